/*
 * aw.h - C ABI of libaw, GB300 (sm_103a) full-polarisation AW-projection
 * gridding and degridding after arXiv:2206.15117 (Skipper, Scaife & Leahy,
 * "A GPU-based Imager with Polarised Primary-beam Correction").
 *
 * General rules
 *   - Every function returns an int status: AW_OK (0) or one of the AW_E*
 *     codes below.  aw_last_error() returns a message for the calling thread.
 *     No C++ exception crosses this boundary.
 *   - Pointers marked "device" are CUDA device pointers on the context's
 *     device; they are owned by the caller (for instance torch tensors) and
 *     must stay valid until the work enqueued on `stream` has finished.
 *     Pointers marked "host" are read before the call returns.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued asynchronously unless stated.
 *   - Opaque handles (aw_ctx, aw_kernel_set, aw_plan, aw_surrogate) are
 *     owned by the library and freed by the matching *_destroy call.
 *   - Threads: a context and the handles used with it serve one host thread
 *     at a time (the context caches cuFFT plans and scratch, a plan its
 *     work queue and graphs); separate contexts may run concurrently.
 *
 * Conventions (shared by every call)
 *   - Grid of N x N uv cells (N a power of two, 16..16384), image cell dl
 *     radians, field F = N dl, uv cell 1/F wavelengths.  Grid index g holds
 *     u = (g - N/2)/F; image pixel q holds l = (q - N/2) dl.  Planes are
 *     stored [npol][N][N], row (v) major, complex64 interleaved (re, im).
 *   - npol = 1: Stokes I, no A term.  npol = 4: visibilities carry the linear
 *     correlations XX, XY, YX, YY; grids and images carry Stokes I, Q, U, V
 *     (Eq. 4 of the paper, with U = (XY + YX)/2).
 *   - Degridding is V = sum I exp(-2 pi i (u l + v m + w (n - 1))) (Eq. 2 with
 *     the usual sign); gridding is its adjoint.
 *   - A visibility with w < 0 is handled at (-u, -v, -w) as P conj(V)
 *     (P swaps XY and YX): the reversed baseline, exact for baseline-averaged
 *     beams (Sec. 3.2) and, with per-baseline kernels, taking the class of
 *     the two antenna types in swapped order.
 */
#ifndef AW_H
#define AW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AW_OK 0
#define AW_EINVAL 1          /* bad argument (null pointer, size, mode)          */
#define AW_ENOMEM 2          /* device or host allocation failed                  */
#define AW_ECUDA 3           /* a CUDA or cuFFT call failed                       */
#define AW_ETIMEOUT 4        /* a bounded device wait gave up                     */
#define AW_EUNSUPPORTED 5    /* valid request this build does not handle          */
#define AW_EREJECTED 6       /* informational: surrogate bins fell back to exact  */

#define AW_ROLE_GRID 0       /* uv transform of psi W ((M^S)'^-1 T): corr -> Stokes */
#define AW_ROLE_DEGRID 1     /* uv transform of psi W* (M T^-1): Stokes -> corr     */
#define AW_ROLE_ADJOINT 2    /* conjugate transpose of the GRID role               */
#define AW_ROLE_BEAM 3       /* conjugate transpose of the DEGRID role: gridding
                              * weighted by the beam (the exact adjoint of
                              * degridding), for UV-domain mosaics (Sec. 2.2)      */

#define AW_STORAGE_FP32 0    /* complex64 tables                                  */
#define AW_STORAGE_BF16 1    /* complex as two bfloat16, FP32 arithmetic          */
#define AW_STORAGE_FP16 2    /* complex as two float16, FP32 arithmetic           */

typedef struct aw_ctx aw_ctx;
typedef struct aw_kernel_set aw_kernel_set;
typedef struct aw_plan aw_plan;
typedef struct aw_surrogate aw_surrogate;

/* ---- kernel specification ---------------------------------------------- */
/*
 * Bins: w plane p (nw planes linear in |w|, centres (p + 1/2) w_max / nw;
 * nw = 1 switches the w term off), parallactic-angle bin a, beam-frequency
 * bin f, and with ntype >= 2 the baseline class k = ti * ntype + tj; bin index
 * ((k * nw + p) * npa + a) * nfb + f.  Sec. 3.2 of the paper averages beams
 * over channel ranges and baselines ("for performance reasons"); these bins
 * are that averaging, and the baseline classes undo the baseline part of it.
 * A visibility flipped to w >= 0 (V -> P conj V) is the reversed baseline and
 * takes class tj * ntype + ti.
 */
typedef struct aw_kernel_spec {
    int32_t N;               /* grid side                                        */
    double dl;               /* image cell, radians                              */
    int32_t OS;              /* oversampling, 1..64; even if a support is odd    */
    double W;                /* PSWF taper support in cells (c = pi W / 2)       */
    int32_t npol;            /* 1 or 4                                           */
    int32_t nw;              /* number of w planes, >= 1                         */
    double w_max;            /* |w| covered by the planes, wavelengths           */
    const int32_t *supports; /* host [nw]: full kernel width S_p per plane, 2..128 */
    int32_t npa;             /* parallactic-angle bins (npol 4), >= 1            */
    const double *pa;        /* host [npa]: bin centres, radians                 */
    int32_t nfb;             /* beam-frequency bins (npol 4), >= 1               */
    const double *fbin_freqs;/* host [nfb]: bin centres, Hz                      */
    double dish_d;           /* dish diameter for the Airy beam, metres          */
    double d_xy[2];          /* leakage X<-Y (re, im)                            */
    double d_yx[2];          /* leakage Y<-X (re, im)                            */
    double eps;              /* Eq. 6 masking fraction (paper: typically 0.2)   */
    int32_t role;            /* AW_ROLE_*                                        */
    int32_t storage;         /* AW_STORAGE_*                                     */
    double point_l, point_m; /* antenna pointing relative to the image phase
                              * centre (direction cosines): the beam is evaluated
                              * at (l - point_l, m - point_m); 0 for a single
                              * pointing, the field offset in UV-domain mosaics   */
    int32_t ntype;           /* antenna types with their own leakage, 0..16; 0 or
                              * 1: every antenna has d_xy, d_yx (baseline-averaged
                              * Mueller kernels, Sec. 3.2).  >= 2: per-baseline
                              * kernels, one class per ordered type pair (ti, tj)
                              * with M = J_ti kron conj(J_tj)                     */
    const double *type_leak; /* host [ntype][4]: d_xy (re, im), d_yx (re, im) per
                              * type; NULL if ntype <= 1                          */
} aw_kernel_spec;

typedef struct aw_kernel_info {
    int64_t bytes;           /* device bytes of the tables                       */
    int32_t nbins;
    int32_t max_support;
    int32_t npol;
    int32_t role;
    int32_t storage;
    int32_t N;
    int32_t OS;
    int32_t n_rejected;      /* surrogate sets: bins that use exact tables       */
} aw_kernel_info;

/* ---- visibilities -------------------------------------------------------- */
typedef struct aw_vis_desc {
    int64_t nvis;
    int64_t nrow;
    int32_t nchan;
    const double *uvw;          /* device f64 [nrow][3], metres                  */
    const uint32_t *row_of_vis; /* device [nvis]                                 */
    const uint16_t *chan_of_vis;/* device [nvis]                                 */
    const double *freq;         /* device f64 [nchan], Hz                        */
    const uint8_t *pa_bin;      /* device [nrow] or NULL (all 0)                 */
    const uint8_t *fbin;        /* device [nchan] or NULL (all 0)                */
    const uint8_t *flags;       /* device [nvis] or NULL; nonzero = flagged      */
    const uint8_t *row_types;   /* device [nrow][2] or NULL: types of the row's two
                                 * antennas, in the order of the baseline the uvw
                                 * belongs to (read only by kernel sets with
                                 * ntype >= 2; NULL means type 0 for both; values
                                 * >= ntype count as ntype - 1)                   */
} aw_vis_desc;

typedef struct aw_tune {
    int32_t tile;            /* grid tile side for the visibility sort, 8..256 (power of 2) */
    int32_t chunk;           /* max visibilities per work item, 32..2048          */
    int32_t ctas_per_sm;     /* persistent launch: CTAs per SM, 1..8              */
    int32_t dg_tile;         /* degridding super-tile side (power of 2, 32..4096);
                              * 0 selects 1024.  Degridding visits visibilities
                              * grouped by (bin, super-tile, oversampled offset) */
    int32_t grid_mode;       /* AW_GRID_TILES, AW_GRID_OFFSETS, AW_GRID_HYBRID or
                              * AW_GRID_REGION                                    */
    int32_t split_planes;    /* AW_GRID_HYBRID: visibilities in w planes
                              * [0, split_planes) take the TILES schedule, the
                              * rest OFFSETS; 0..nw.  Ignored by the other modes */
} aw_tune;

/* Gridding schedules (aw_tune.grid_mode).  TILES: work items of one bin and
 * one grid tile, register accumulation per residue class of the support,
 * persistent launch (tile, chunk, ctas_per_sm apply).  OFFSETS: the
 * degridding items (one bin, super-tile and oversampled offset), each kernel
 * tap loaded once per item and added for every visibility with vector
 * atomics (dg_tile applies).  HYBRID: the low w planes (the small supports,
 * split_planes of them) on TILES and the others on OFFSETS, the two kernels
 * running at the same time on two streams (the plan owns the second stream;
 * the call forks from and joins back into the caller's stream, also inside
 * the graph of aw_grid_batched).  The TILES kernel is bound by the L2->SM
 * stream of kernel values, the OFFSETS kernel by its atomics, so sharing the
 * SMs between them beats either alone.  REGION: work items of one bin and
 * one grid tile whose side is chosen per support, sorted by oversampled
 * offset; the CTA accumulates the tile's output region (tile + support - 1
 * cells square, at most 56) in shared memory, each thread holding kernel
 * taps in registers for all visibilities of an offset (full-pol: one tap's 16
 * Mueller values; Stokes I: up to 18 taps of one value), and adds the region to
 * the grid once; bins of planes from split_planes on, and bins whose support
 * has no region form (above 49 cells; full-pol: rows that do not split into
 * passes of 32 taps over 4-10 warps; Stokes I: not a multiple of 4), take
 * OFFSETS on the plan's second stream at the same time.  All modes give the
 * same grid up to FP32 rounding order. */
enum { AW_GRID_TILES = 0, AW_GRID_OFFSETS = 1, AW_GRID_HYBRID = 2, AW_GRID_REGION = 3 };

typedef struct aw_plan_info {
    int64_t nvis;
    int64_t nvalid;          /* visibilities that are gridded                     */
    int64_t n_outside;       /* skipped: footprint not inside the grid            */
    int64_t n_flagged;       /* skipped: flagged                                  */
    int64_t nitems;          /* work items                                        */
    int32_t tile;
    int32_t chunk;
    double mean_taps;        /* mean S^2 over the valid visibilities              */
    int64_t nitems_degrid;   /* degridding work items                             */
    int32_t grid_kernels;    /* kernels one aw_grid / aw_grid_batched call launches */
    int32_t region_lists;    /* AW_GRID_REGION: supports on the region kernel      */
} aw_plan_info;

typedef struct aw_stats {
    int64_t n_gridded;
    int64_t n_outside;
    int64_t n_flagged;
    int64_t n_nonfinite;     /* skipped at grid time: NaN/Inf value or weight     */
    double weight_sum;       /* sum over gridded vis of the mean correlation weight */
} aw_stats;

/* ---- context --------------------------------------------------------------- */

/* Message of the last failing call on this thread ("" if none). */
const char *aw_last_error(void);

/* Create a context on CUDA device `device` (cuFFT plan cache, scratch,
 * device status word).  *ctx receives the handle. */
int aw_create(aw_ctx **ctx, int device);
int aw_destroy(aw_ctx *ctx);

/* ---- kernel synthesis (Sec. 3.2, Sec. 3.3, Eq. 2-6) ------------------------ */

/*
 * aw_make_kernels - build the oversampled convolution kernels of every bin.
 *
 * Paper: Sec. 3.2 (degridding kernels are the FFT of the Mueller-matrix cells
 * of Eq. 5 after the anti-aliasing function and the w term; gridding kernels
 * come from the inverse Mueller matrix) and Sec. 3.3 / Eq. 6 (the diagonal of
 * a copy of M^S is regularised before inversion).  For every bin: the image
 * function (taper psi(l) psi(m) x w term x Mueller cell) is sampled on M x M
 * points over the field (M the smallest power of two >= 2 S_p, >= 16; the
 * l = -F/2 row and column set to 0), zero-padded to (M OS)^2, transformed
 * with a double-precision FFT, scaled by 1/M^2 and cut to S_p x S_p taps at
 * OS x OS fine offsets.  Canonical table order per bin (aw_kernel_set_import
 * and _export): [OS][OS][S][S][npol*npol], Mueller index out * npol + in;
 * inside the library the values of one (bin, offset) block are stored in
 * 16-byte chunks, chunk-major and tap-minor, for coalesced loads.  A visibility at oversampled coordinate Xi
 * covers cells x0..x0+S-1, x0 = floor((Xi - rho)/OS), rho = (S-2) OS/2; tap j
 * holds the kernel at j OS - rho - fx oversampled units (fx the fine offset).
 * Mueller algebra per pixel in FP64: J = E(r) [[1, d_xy], [d_yx, 1]] R(chi),
 * E = 2 J1(x)/x (Airy), M = J (x) conj(J), M^S = T M T^-1.
 *
 * Runs on `stream`; the call returns once the tables are built (it
 * synchronises `stream`).  The set is owned by the library.
 * Errors: AW_EINVAL for a bad spec (N not a power of two, OS out of range,
 * odd support with odd OS, npol not 1/4, null arrays), AW_ENOMEM, AW_ECUDA.
 */
int aw_make_kernels(aw_ctx *ctx, const aw_kernel_spec *spec, aw_kernel_set **out, void *stream);

/*
 * aw_kernel_set_import - build a set from caller tables (for instance tables
 * evaluated by a surrogate or computed elsewhere).  `tables` is a device
 * complex64 array holding every bin's block in the layout above, bins
 * consecutive; it is converted to spec->storage.  spec->role is recorded.
 */
int aw_kernel_set_import(aw_ctx *ctx, const aw_kernel_spec *spec, const void *tables,
                         aw_kernel_set **out, void *stream);

/* Copy bin `bin`'s table as complex64 (converted from the storage type) to
 * device memory `dst` ([OS][OS][S][S][P] complex64). */
int aw_kernel_set_export(const aw_kernel_set *kset, int32_t bin, void *dst, void *stream);
int aw_kernel_set_info(const aw_kernel_set *kset, aw_kernel_info *info);

/*
 * Kernel-set cache on disk.  aw_kernel_spec_hash - a 64-bit key of `spec`:
 * FNV-1a 64 of a canonical little-endian encoding of the spec after the
 * library's own validation and normalisation (every field and array that
 * defines the tables; AW_EINVAL for an invalid spec).  aw_kernel_set_save -
 * write `kset` to `path`: magic "AWKSET01", that spec encoding, the table
 * scale, the rejected-bin count and the table size, a header checksum, then
 * the tables in their storage format and layout and a checksum of them
 * (streamed through host memory in 256 MiB pieces; synchronises the device).
 * aw_kernel_set_load - a new set on ctx's device from such a file (*out, freed
 * with aw_kernel_set_destroy): the same geometry, tables and scale.  AW_EINVAL
 * (and *out = NULL) if the file is missing, truncated, has trailing bytes, a
 * bad magic or checksum, or tables whose size does not match its spec.
 */
int aw_kernel_spec_hash(const aw_kernel_spec *spec, uint64_t *hash);
int aw_kernel_set_save(const aw_kernel_set *kset, const char *path);
int aw_kernel_set_load(aw_ctx *ctx, const char *path, aw_kernel_set **out);
int aw_kernel_set_destroy(aw_kernel_set *kset);

/* ---- plan: coordinates (FP64) and device key sort --------------------------- */

/*
 * aw_plan_create - per-visibility coordinates and the sorted work list.
 *
 * Paper: the baseline of Eq. 2 is in wavelengths; Sec. 2.1 (w-projection with
 * a configurable number of w planes).  For each visibility, in FP64 with a
 * fixed operation order and no fused multiply-add: f = freq/c,
 * (u, v, w) = uvw f, flip if w < 0, X = u N dl OS + (N/2) OS, Xi = floor(X +
 * 1/2), w plane floor(|w| nw / w_max) clamped, bin, footprint start x0 and
 * fine offset fx as in aw_make_kernels.  A visibility is gridded only if its
 * whole footprint lies inside the grid and it is not flagged.  The valid
 * visibilities are sorted on the device (LSD radix sort: per-digit
 * histogram, exclusive scan, stable scatter) by (bin, tile of tune->tile
 * cells, position in tile) and cut into work items of at most tune->chunk.
 * The plan depends on the kernel set only through N, OS, the bins and their
 * supports; any set with the same geometry may be used with it.
 * tune == NULL uses the last aw_autotune result of this context (its cache),
 * or tile 32, chunk 256 if the context has none; a cached HYBRID tune whose
 * split_planes is not inside 1..nw-1 of this kernel set is used with the
 * OFFSETS schedule instead, as is a cached REGION tune whose split_planes is
 * above this set's nw.  Synchronises `stream`.
 */
int aw_plan_create(aw_ctx *ctx, const aw_vis_desc *vis, const aw_kernel_set *kset,
                   const aw_tune *tune, aw_plan **out, void *stream);
int aw_plan_query(const aw_plan *plan, aw_plan_info *info);
int aw_plan_destroy(aw_plan *plan);

/*
 * aw_plan_coords - the plan's integer coordinates in the caller's visibility
 * order (device outputs, each [nvis]; any may be NULL): footprint start x0,
 * y0, fine offsets fx, fy, bin, flip (0/1) and valid (0/1).  For checking.
 */
int aw_plan_coords(const aw_plan *plan, int32_t *x0, int32_t *y0, int32_t *fx, int32_t *fy,
                   int32_t *bin, uint8_t *flip, uint8_t *valid, void *stream);

/* aw_plan_order - the sorted order: perm[i] = caller index of the i-th
 * visibility (device [nvis]; valid ones first, in key order). */
int aw_plan_order(const aw_plan *plan, uint32_t *perm, void *stream);

/* ---- gridding and degridding (the hot path) -------------------------------- */

/*
 * aw_grid - convolve visibilities onto the uv grid (Sec. 3.2 gridding stage).
 *
 *   G[s][y0+jy][x0+jx] += sum_c K[bin][fy][fx][jy][jx][s npol + c] w'_c V'_c
 *
 * vis: device complex64 [nvis][npol] in the caller's order; weight: device
 * float [nvis][npol] or NULL (all 1); grid: device complex64 [npol][N][N],
 * ACCUMULATED into (the caller zeroes it).  Visibilities with a NaN/Inf value
 * or weight are skipped and counted.  FP32 products and sums; the summation
 * order of overlapping footprints is not fixed (atomics).  kset must have
 * role AW_ROLE_GRID (or any role, used as given).  If stats != NULL (host),
 * the call synchronises `stream` and fills it.
 */
int aw_grid(aw_ctx *ctx, const aw_plan *plan, const aw_kernel_set *kset, const void *vis,
            const float *weight, void *grid, aw_stats *stats, void *stream);

/*
 * aw_degrid - gather a model grid into visibilities (Sec. 3.2 degridding).
 *
 *   V'_c = sum_s sum_taps K[bin][fy][fx][jy][jx][c npol + s] G[s][y0+jy][x0+jx]
 *
 * then V = P conj(V') for flipped visibilities.  grid: device complex64
 * [npol][N][N]; vis_out: device complex64 [nvis][npol] in the caller's order,
 * OVERWRITTEN (zero for visibilities the plan does not grid).  Visibilities
 * that share a bin, a super-tile and an oversampled offset share one kernel
 * block staged in shared memory; FP32 products, warp reductions.
 */
int aw_degrid(aw_ctx *ctx, const aw_plan *plan, const aw_kernel_set *kset, const void *grid,
              void *vis_out, void *stream);

/*
 * aw_grid_batched - aw_grid as one launch over all the plan's work items
 * (every channel, polarisation and w plane of uneven counts in one launch),
 * captured once in a CUDA graph and replayed.  With grid_mode TILES the
 * launch is persistent over a work queue, ctas_per_sm from the plan's tune.
 * The plan caches the graphs of the last two (vis, weight, grid, kset,
 * stream) argument sets (a double-buffered caller alternates between two
 * without re-capturing); do not call it for one plan from two threads.
 * Same result as aw_grid within FP32 summation-order rounding.
 */
int aw_grid_batched(aw_ctx *ctx, aw_plan *plan, const aw_kernel_set *kset, const void *vis,
                    const float *weight, void *grid, aw_stats *stats, void *stream);

/*
 * aw_autotune - time aw_grid_batched over candidate (tile, chunk,
 * ctas_per_sm) of the TILES schedule, two super-tile sizes of the OFFSETS
 * schedule and up to three split planes (the first planes holding about 25,
 * 35 and 45 % of the visibility-taps) at 2 or 3 TILES CTAs per SM of the
 * HYBRID schedule on the given visibilities (pass a subsample to keep it
 * short) and return the fastest in *out; it is also kept in the context as the tune
 * aw_plan_create uses when given NULL.  Uses a scratch grid it allocates.
 * Synchronises `stream`.
 */
int aw_autotune(aw_ctx *ctx, const aw_vis_desc *vis, const aw_kernel_set *kset, aw_tune *out,
                void *stream);

/* ---- uv grid -> image (Sec. 2.2: FFT on the GPU) ---------------------------- */

/*
 * aw_fft_to_image - dirty image planes from uv grid planes.
 *
 *   I(q) = sum_g G(g) exp(+2 pi i (g - N/2)(q - N/2)/N) / (c(qx) c(qy)) / weight_sum
 *
 * real part, c(q) = psi(2 l_q / F) the taper (grid correction); row/column 0
 * are written as 0.  grid (device complex64 [npol][N][N], kset's N and npol)
 * is used as FFT scratch and left transformed; image: device float
 * [npol][N][N].  cuFFT (FP32 complex) plus the library's own shift and
 * grid-correction kernels.
 */
int aw_fft_to_image(aw_ctx *ctx, const aw_kernel_set *kset, void *grid, double weight_sum,
                    float *image, void *stream);

/* ---- learned kernel surrogate --------------------------------------------- */
/*
 * A SIREN-style coordinate MLP standing in for the per-bin FFT kernel
 * synthesis of Sec. 3.2: it maps the continuous coordinates of a tap
 * (grid-minus-visibility offset d_u, d_v in cells, w in wavelengths,
 * frequency, parallactic angle) to the npol^2 complex Mueller kernel values
 * of that tap, and is trained on tables built by aw_make_kernels.
 *   features x = [d_u/s, d_v/s, 2 w/w_max - 1, (f - f_c)/f_h, (chi - chi_c)/chi_h],
 *   s = D (S(w)/2 + 1), S(w) = norm_supports[min(floor(w norm_nw / w_max),
 *   norm_nw - 1)]: offsets in units of the half support of the w plane that
 *   |w| falls in, for one fixed plane layout shared by training and use
 *   layers [5, width x n_hidden, 2 npol^2]; hidden h = sin(omega0 (W h + b)),
 *   linear output; kernel value = output * out_scale.
 *   Parameters: one flat FP32 vector, per layer W [out][in] then b [out].
 *   Loss (1/B) sum (y - t)^2; Adam (b1 0.9, b2 0.999, eps 1e-8) with bias
 *   correction and a cosine learning-rate decay from lr to lr_final.
 * Training runs in the library's kernels with FP32 master weights (on the
 * tensor cores for width 128: aw_surrogate_set_train_engine); the inline
 * evaluation uses an FP16 copy of the weights with FP32 accumulation.
 */
typedef struct aw_surrogate_cfg {
    int32_t npol;            /* 1 or 4                                           */
    int32_t width;           /* hidden width (128)                               */
    int32_t n_hidden;        /* number of sine layers (4)                        */
    float omega0;            /* SIREN frequency (30)                             */
    double D, w_max, f_c, f_h, chi_c, chi_h;  /* feature scales (see above)      */
    float out_scale;         /* kernel value = output * out_scale                */
    uint64_t seed;           /* initialisation seed                              */
    int32_t norm_nw;         /* planes of the offset-normalisation layout, 1..256 */
    const int32_t *norm_supports;  /* host [norm_nw]: support per plane (copied) */
} aw_surrogate_cfg;

typedef struct aw_train_cfg {
    int32_t steps;           /* Adam steps                                        */
    int32_t batch;           /* points per step (sampled from the exact tables)   */
    float lr, lr_final;      /* cosine decay from lr to lr_final                  */
    uint64_t seed;           /* sampling seed (SplitMix64 counters)               */
} aw_train_cfg;

typedef struct aw_train_report {
    float loss_first;        /* loss of the first step                            */
    float loss_last;         /* mean loss over the last 5 % of steps              */
    int32_t steps;
    double seconds;          /* wall time of the training loop                    */
} aw_train_report;

int aw_surrogate_create(aw_ctx *ctx, const aw_surrogate_cfg *cfg, aw_surrogate **out);
int aw_surrogate_destroy(aw_surrogate *sur);
int aw_surrogate_nparams(const aw_surrogate *sur, int64_t *n);
/* Copy parameters from / to host memory ([nparams] FP32).  set_params also
 * resets the Adam state. */
int aw_surrogate_set_params(aw_surrogate *sur, const float *host_params);
int aw_surrogate_get_params(const aw_surrogate *sur, float *host_params);
/* Forward pass on B feature rows: X device float [B][5] -> Y device float
 * [B][2 npol^2] (FP32 weights). */
int aw_surrogate_forward(aw_ctx *ctx, aw_surrogate *sur, const float *X, int32_t B, float *Y, void *stream);
/* Loss and gradient on one batch (targets T device float [B][2 npol^2]):
 * *loss (host) and grad (device float [nparams]).  Synchronises `stream`. */
int aw_surrogate_loss_grad(aw_ctx *ctx, aw_surrogate *sur, const float *X, const float *T, int32_t B,
                           double *loss, float *grad, void *stream);
/* Train on random (bin, fine offset, tap) points of `exact` (its role and
 * npol must match the surrogate).  The network has no baseline-class input:
 * a set with ntype >= 2 returns AW_EUNSUPPORTED here, in aw_surrogate_tables
 * and in aw_grid_learned.  Synchronises `stream`. */
int aw_surrogate_train(aw_ctx *ctx, aw_surrogate *sur, const aw_kernel_set *exact, const aw_train_cfg *cfg,
                       aw_train_report *report, void *stream);
/*
 * aw_surrogate_tables - evaluate the surrogate at every table point of
 * `exact` into a new set with the same geometry (`storage` must equal the
 * exact set's storage, else AW_EUNSUPPORTED).  Per w
 * plane, if the relative L2 error of any of its bins exceeds reject_rel the
 * plane keeps the exact tables (fallback; info.n_rejected counts those bins,
 * and the call returns AW_EREJECTED if any).  bin_err (host [nbins], may be
 * NULL) receives each bin's relative L2 error.  Synchronises `stream`.
 */
int aw_surrogate_tables(aw_ctx *ctx, aw_surrogate *sur, const aw_kernel_set *exact, float reject_rel,
                        int32_t storage, aw_kernel_set **out, float *bin_err, void *stream);

/*
 * aw_grid_learned - gridding with the surrogate evaluated inline (no kernel
 * tables): for every visibility and tap of its footprint the MLP runs on
 * tensor cores (FP16 weights and activations, FP32 accumulation; engine
 * chosen by aw_surrogate_set_engine) at the tap's exact offset from the
 * visibility (no oversampling grid), the
 * visibility's exact |w| (no w-plane quantisation), its beam-frequency bin centre
 * and its parallactic-angle bin centre; the P kernel values are applied as
 * in aw_grid (same flip, weights, skip rules, accumulation into `grid`).
 * The plan gives the footprints (supports per w plane) and the order.  W
 * planes rejected by the last aw_surrogate_tables call use `fallback` (the
 * exact set) at the plan's quantised offsets.  The surrogate must have width
 * 128 and 4 sine layers (AW_EUNSUPPORTED otherwise).  The plan's visibility
 * descriptor arrays are read again and must still be valid.  With the
 * TCGEN05 engine the call synchronises `stream` and returns AW_ETIMEOUT if a
 * bounded tensor-core completion wait gave up (grid invalid).
 */
int aw_grid_learned(aw_ctx *ctx, const aw_plan *plan, aw_surrogate *sur, const aw_kernel_set *fallback,
                    const void *vis, const float *weight, void *grid, aw_stats *stats, void *stream);

/*
 * aw_degrid_learned - degridding with the surrogate evaluated inline: for
 * every valid visibility of the plan and every tap of its footprint the
 * network (trained on a DEGRID-role set) gives the Mueller kernel K_{c,s} at
 * the tap's exact offset, exact |w|, frequency (aw_surrogate_set_freq_mode)
 * and PA bin centre, as in aw_grid_learned; vis_out[c] = sum over taps and s
 * of K_{c,s} model_s[cell], then P conj() for flipped visibilities, as in
 * aw_degrid.  Invalid visibilities get 0.  W planes rejected by the last
 * aw_surrogate_tables call use `fallback` (the exact set, role DEGRID or
 * ADJOINT, AW_EINVAL otherwise) at the plan's quantised offsets.  model:
 * device complex64 [npol][N][N]; vis_out: device complex64 [nvis][npol],
 * overwritten.  Runs on the TCGEN05 engine only (AW_EUNSUPPORTED with
 * MMA_SYNC); synchronises `stream`; AW_ETIMEOUT if a bounded tensor-core
 * completion wait gave up (vis_out invalid).
 */
int aw_degrid_learned(aw_ctx *ctx, const aw_plan *plan, aw_surrogate *sur, const aw_kernel_set *fallback,
                      const void *model, void *vis_out, void *stream);

/*
 * aw_surrogate_set_engine - tensor-core generation of the inline evaluation in
 * aw_grid_learned.  AW_ENGINE_TCGEN05 (default): 128-row tiles per CTA,
 * tcgen05.mma with FP32 accumulators in tensor memory, one thread issuing.
 * AW_ENGINE_MMA_SYNC: 16-row tiles per warp on mma.sync.m16n8k16.  Both give
 * the same result up to FP32 summation order and the FP16 rounding of the
 * activations.  AW_EINVAL for any other value.
 */
enum { AW_ENGINE_MMA_SYNC = 0, AW_ENGINE_TCGEN05 = 1 };
int aw_surrogate_set_engine(aw_surrogate *sur, int32_t engine);

/*
 * aw_surrogate_set_train_engine - where the products of a training step (and
 * of aw_surrogate_loss_grad) run.  AW_TRAIN_TCGEN05 (default): for a network
 * of width 128 with at least 2 hidden layers, every layer but the first as
 * tcgen05.mma (FP16 operands: activations, weights, output errors; FP32
 * accumulation, FP32 master weights and Adam), the weight gradients as
 * GEMMs over the batch; the batch must be a multiple of 128.  Other shapes
 * fall back to AW_TRAIN_FP32.  AW_TRAIN_FP32: FP32 tiled GEMMs on the CUDA
 * cores.  The network is Sec. 3.2's kernel synthesis stood in for by a
 * coordinate MLP (see aw_surrogate_create).  AW_EINVAL for another value.
 */
enum { AW_TRAIN_FP32 = 0, AW_TRAIN_TCGEN05 = 1 };
int aw_surrogate_set_train_engine(aw_surrogate *sur, int32_t engine);

/*
 * aw_surrogate_set_freq_mode - the frequency the inline evaluation of
 * aw_grid_learned feeds the network.  AW_FREQ_BIN (default): the centre of
 * the visibility's beam-frequency bin, as the exact tables average the beam
 * over the bin's channels (Sec. 3.2).  AW_FREQ_CHANNEL: the visibility's own
 * channel frequency, which removes the channel averaging without any table
 * memory (the network must have been trained over the band).  Rejected
 * planes use the exact tables in either mode.  AW_EINVAL for other values.
 */
enum { AW_FREQ_BIN = 0, AW_FREQ_CHANNEL = 1 };
int aw_surrogate_set_freq_mode(aw_surrogate *sur, int32_t mode);

/*
 * aw_surrogate_save - write the surrogate to the file `path` (created or
 * truncated): its configuration, FP32 parameters, the per-w-plane rejection
 * of the last aw_surrogate_tables call, the engine and the frequency mode.  Every field is
 * little-endian with no padding, after the 8-byte magic "AWSURR01", and the
 * file ends with an FNV-1a 64 checksum of the bytes before it; the layout is
 * the same on every host.  Adam moments are not saved.  Synchronises the
 * device.  AW_EINVAL if the file cannot be written.
 *
 * aw_surrogate_load - create a surrogate on ctx's device from such a file
 * (*out, freed with aw_surrogate_destroy).  Training continues from the
 * loaded parameters with fresh Adam moments.  AW_EINVAL (and *out = NULL) if
 * the file is missing, truncated, has trailing bytes, a bad magic or
 * checksum, or a parameter count that does not match its configuration.
 */
int aw_surrogate_save(const aw_surrogate *sur, const char *path);
int aw_surrogate_load(aw_ctx *ctx, const char *path, aw_surrogate **out);

/* ---- mosaic weighting (Sec. 2.2, Eq. 1) ------------------------------------- */

/*
 * mosaic_gamma - gamma(l, m) = [sqrt(sum B_i^2) / max sqrt(sum B_i^2)]_pbp x
 * [1 / sum B_i^2]_wc (Eq. 1), set to 0 where the pbp factor is below eps.
 * beams: device float [nfield][N][N]; gamma: device float [N][N].  Uses a
 * context scratch word for the maximum.
 */
int mosaic_gamma(aw_ctx *ctx, const float *beams, int32_t nfield, int32_t N, float eps,
                 float *gamma, void *stream);

/*
 * mosaic_gamma_noalloc - mosaic_gamma for callers that cannot allocate device
 * memory: code inside a framework whose caching allocator owns the device
 * memory (a second allocator fragments it), real-time loops that forbid
 * allocation after start-up (cudaMalloc may synchronise and takes unbounded
 * time).  It needs no aw_ctx (aw_create allocates) and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 * The paper has no counterpart; this is a deployment variant of the Eq. 1 call
 * above, with the same arguments and result.
 *
 * Scratch: a fixed file-scope device array of 4097 floats (16 KB) inside
 * libaw, held by every GPU that loads the library until the process exits.
 * Limit: N * N <= 4096 * 4096 pixels; larger images return AW_EINVAL before
 * any GPU work.  The first call on a device (and the first after its context
 * is re-created, e.g. by cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call shares the one
 * array and
 * nothing in it needs to start at zero (each pass reads only slots written
 * earlier in the same call), but calls whose GPU work overlaps (different
 * streams or host threads) race on it: serialise them.  beams: device float
 * [nfield][N][N]; gamma: device float [N][N]; work is enqueued on `stream`.
 */
int mosaic_gamma_noalloc(const float *beams, int32_t nfield, int32_t N, float eps, float *gamma,
                         void *stream);

/* ---- image-domain mosaics: reprojection and combination ----------------------
 *
 * Sec. 2.2: each mosaic field is imaged at its own phase centre; image-plane
 * reprojection brings the images to a common phase position to form the
 * mosaic, and the model is reprojected back to each field before degridding.
 * Readings: frames are orthographic (SIN) projections about a phase centre
 * (ra0, dec0), with l = cos dec sin(ra - ra0), m = sin dec cos dec0 -
 * cos dec sin dec0 cos(ra - ra0); pixel (qx, qy) of a frame sits at
 * l = (qx - cx) dl, m = (qy - cy) dl.  An output pixel is carried to the
 * source frame (FP64; the map between two frames is a rotation of
 * (l, m, n)), and the source image is interpolated there: bilinear (2 x 2)
 * or Keys cubic convolution, a = -1/2 (4 x 4), in FP32.  Where the stencil
 * leaves the source image, or the direction is off the visible hemisphere of
 * either frame, the output is `fill`.
 */
typedef struct aw_sky_frame {
    double ra0, dec0;        /* phase centre, radians                              */
    double dl;               /* pixel size, direction-cosine units (> 0)           */
    double cx, cy;           /* pixel of the phase centre                          */
    int32_t N;               /* image side (N x N pixels)                          */
    int32_t reserved;
} aw_sky_frame;

enum { AW_INTERP_BILINEAR = 0, AW_INTERP_CUBIC = 1 };

/*
 * aw_reproject - src: device float [nplane][src->N][src->N]; dst: device
 * float [nplane][dst->N][dst->N], overwritten; the planes share the pixel
 * mapping.  Frames are host structs.
 */
int aw_reproject(aw_ctx *ctx, const float *src, const aw_sky_frame *src_frame, float *dst,
                 const aw_sky_frame *dst_frame, int32_t nplane, int32_t interp, float fill, void *stream);

/*
 * aw_mosaic_combine - Eq. 1 on images already in the common frame:
 * out[p] = gamma * sum_f beams[f] * images[f][p].  images: device float
 * [nfield][nplane][N][N]; beams: device float [nfield][N][N]; gamma: device
 * float [N][N] (mosaic_gamma); out: device float [nplane][N][N].
 */
int aw_mosaic_combine(aw_ctx *ctx, const float *images, const float *beams, const float *gamma, int32_t nfield,
                      int32_t nplane, int32_t N, float *out, void *stream);

/*
 * aw_phase_rotate - move visibilities to a new phase centre: each field of a
 * UV-domain mosaic (Sec. 2.2) is gridded about the mosaic's centre.  The
 * baselines are unchanged; their components about the new centre are
 * uvw' = B_to B_from^T uvw (B: rows east, north, centre of a frame), and with
 * the degridding convention V = sum I exp(-2 pi i (u l + v m + w (n - 1))) the
 * visibilities become V' = V exp(2 pi i (w' - w) nu / c).  Rotation and phase
 * in FP64, the product in FP32.  vd: the observation (uvw metres, rows,
 * channels, frequencies; device arrays); uvw_out: device f64 [nrow][3] or NULL
 * (must not alias vd->uvw: the phases read the input uvw); vis, vis_out:
 * device complex64 [nvis][npol] (may alias).  Centres (ra, dec) in radians.
 */
int aw_phase_rotate(aw_ctx *ctx, const aw_vis_desc *vd, double *uvw_out, const void *vis, void *vis_out, int32_t npol,
                    double ra_from, double dec_from, double ra_to, double dec_to, void *stream);

/* ---- cleaning: Cotton-Schwab major cycles, Hogbom minor cycle ---------------
 *
 * Sec. 2.1: the imager cleans with the Cotton-Schwab algorithm, controlled by
 * the number of clean cycles, the loop gain, the cycle factor and a threshold;
 * Sec. 4 names Hogbom cleaning as the iterative part.  A major cycle grids the
 * residual visibilities, makes the residual image, runs the minor cycle on it,
 * predicts the model (image -> grid -> degrid) and subtracts it from the
 * observed visibilities.  Readings (the paper does not write the steps out):
 * the minor cycle picks the peak of |I| in the clean window (ties to the
 * lowest row-major pixel index), takes gain x the residual of every Stokes
 * plane there as the component, and subtracts it with a square patch of the
 * point-spread function of half-width patch_half, in FP32 with one rounding
 * per multiply and per subtraction; the cycle threshold is max(threshold,
 * cycle_factor * sidelobe * peak); the point-spread function is the Stokes I
 * image of unit Stokes I visibilities, divided by its value at the phase
 * centre; sidelobe is its largest |value| outside the main lobe, a disk of
 * radius r0 = the first x > 0 with psf[N/2][N/2 + x] <= 0, and within N/4
 * pixels of the centre on both axes (with A-projection the outer image of
 * unit visibilities carries the inverse beam and the grid correction).
 */
typedef struct aw_clean_cfg {
    int32_t n_major;         /* major cycles, >= 1                                */
    int32_t max_minor;       /* Hogbom iterations per major cycle, >= 0           */
    float gain;              /* loop gain, (0, 1]                                 */
    float threshold;         /* stop when the peak |I| of the residual is below   */
    float cycle_factor;      /* see above; >= 0                                   */
    int32_t patch_half;      /* point-spread-function patch half-width, [0, N/2)  */
    int32_t window[4];       /* clean window x0, y0, x1, y1 (half-open), inside
                              * the image; all zero selects the inner half       */
} aw_clean_cfg;

typedef struct aw_clean_report {
    int32_t n_major;         /* major cycles that ran a minor cycle               */
    int32_t n_minor;         /* Hogbom iterations over all cycles                 */
    float peak_first;        /* peak |I| in the window of the first residual image */
    float peak_last;         /* the same for the final residual image             */
    float sidelobe;          /* point-spread-function sidelobe level              */
    float reserved;
    double weight_sum;       /* sum of the gridding weights (aw_stats.weight_sum) */
} aw_clean_report;

/*
 * aw_image_to_grid - model image -> uv grid for degridding (the adjoint of the
 * image step of aw_fft_to_image): divide by the grid correction (zero on row
 * and column 0), then G(g) = sum_q I(q) exp(-2 pi i (g - N/2)(q - N/2) / N) per
 * plane, no scaling.  image: device float [npol][N][N]; grid: device complex64
 * [npol][N][N], overwritten.  kset supplies N, npol and the taper width.
 */
int aw_image_to_grid(aw_ctx *ctx, const aw_kernel_set *kset, const float *image, void *grid, void *stream);

/*
 * aw_degrid_subtract - vis_out = vis - aw_degrid(grid): the residual
 * visibilities of a major cycle in one pass.  vis, vis_out: device complex64
 * [nvis][npol] in the caller's order; vis_out may be vis.  Visibilities the
 * plan does not grid keep vis.
 */
int aw_degrid_subtract(aw_ctx *ctx, const aw_plan *plan, const aw_kernel_set *kset, const void *grid,
                       const void *vis, void *vis_out, void *stream);

/*
 * aw_psf_sidelobe - the sidelobe level defined above.  psf: device float
 * [N][N]; *sidelobe: host.  Synchronises `stream`.
 */
int aw_psf_sidelobe(aw_ctx *ctx, const float *psf, int32_t N, float *sidelobe, void *stream);

/*
 * aw_hogbom - Hogbom minor cycle (readings above) until the peak |I| in the
 * window is below `threshold` or max_iter components are taken.  residual:
 * device float [npol][N][N], updated in place; psf: device float [N][N] with
 * its peak at (N/2, N/2); model: device float [npol][N][N], components added;
 * window: host int32[4] (x0, y0, x1, y1, half-open, non-empty, inside the
 * image).  One cooperative grid (one or two blocks per SM) runs the loop with
 * three grid barriers per iteration; the peak search keeps the maximum of each
 * 64 x 64 tile (or larger, at most 64 x 64 tiles) and rescans only the tiles a
 * subtraction touched.  Barrier waits are bounded: AW_ETIMEOUT if one gives
 * up (results invalid).  *n_iter: host.  Synchronises `stream`.
 */
int aw_hogbom(aw_ctx *ctx, float *residual, const float *psf, int32_t npol, int32_t N, float gain,
              float threshold, int32_t max_iter, int32_t patch_half, const int32_t *window, float *model,
              int32_t *n_iter, void *stream);

/*
 * aw_clean - Cotton-Schwab cleaning of the plan's visibilities.  kgrid /
 * kdegrid: the plan's GRID and DEGRID kernel sets; vis: device complex64
 * [nvis][npol]; weight: device float [nvis][npol] or NULL.  Outputs (device,
 * overwritten): model float [npol][N][N], residual float [npol][N][N] (the
 * residual image after the last cycle), psf float [N][N].  report: host.
 * Allocates, and frees before returning, one visibility-sized buffer and one
 * grid.  Major cycle: stop if the residual peak is below cfg->threshold,
 * otherwise aw_hogbom down to the cycle threshold, then aw_image_to_grid and
 * aw_degrid_subtract.  Gridding goes through aw_grid_batched (the plan's
 * cached graph).  Synchronises `stream` once per major cycle.
 */
int aw_clean(aw_ctx *ctx, aw_plan *plan, const aw_kernel_set *kgrid, const aw_kernel_set *kdegrid,
             const void *vis, const float *weight, const aw_clean_cfg *cfg, float *model, float *residual,
             float *psf, aw_clean_report *report, void *stream);

/* ---- failure injection and self-tests ------------------------------------- */
/*
 * aw_debug_fail_alloc - failure injection on the host: n >= 0 makes the n-th
 * device allocation of the library from now (0 = the next) fail as if the
 * device were out of memory, once; the call that made it returns AW_ENOMEM
 * and frees what it had allocated.  n = -1 disarms.  Process-wide.
 *
 * aw_debug_alloc_stats - device buffers the library holds now (*live) and
 * device allocations it has attempted since the process started (*calls).
 *
 * aw_debug_wait_timeout - run one of the library's bounded device waits
 * against a condition that never becomes true, on `stream`: which = 0, the
 * grid barrier of the cooperative Hogbom kernel (one block waits for a second
 * arrival); which = 1, the mbarrier completion wait of the tensor-core
 * kernels (an mbarrier that nothing arrives on).  Returns AW_ETIMEOUT when the
 * wait gave up as designed (the barrier after about 9 s, the mbarrier after
 * about 1 s on GB300), AW_OK if it did not;
 * the context stays usable.  Synchronises `stream`.
 */
int aw_debug_fail_alloc(int64_t n);
int aw_debug_alloc_stats(int64_t *live, int64_t *calls);
/*
 * aw_debug_bounds_status - in a library built with -DAW_BOUNDS_CHECK, where
 * the gridding and degridding kernels check every grid, table, shared-memory,
 * record and output index (a bad one is skipped and recorded): *status = the
 * code of the first failed check since the last reset, 0 if none (1-4 tile
 * gridding: grid, table, shared memory, record; 5-8 the same for the offset
 * schedule; 9-13 degridding: table source, shared-memory destination, grid,
 * partial sums, record); reset != 0 clears it.  Synchronises the device.
 * AW_EUNSUPPORTED in a normal build.
 */
int aw_debug_bounds_status(uint32_t *status, int32_t reset);
int aw_debug_wait_timeout(aw_ctx *ctx, int32_t which, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* AW_H */
