// Image-domain mosaics (arXiv:2206.15117 Sec. 2.2): image-plane reprojection
// between phase centres and the Eq. 1 combination.
//
// Reprojection: one thread per destination pixel.  The pixel's direction
// cosines (l, m, n) in the destination frame are rotated into the source
// frame with one 3x3 matrix (the product of the two frames' orthonormal
// axes, formed on the host in FP64), so no trigonometric function is
// evaluated per pixel; the source position and its floor are FP64, the
// interpolation weights and the interpolation FP32 over all planes.
#include <cmath>
#include <new>

#include "aw_internal.h"

namespace {

inline cudaStream_t S_(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int use_device(int dev) {
    int cur = -1;
    AW_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != dev) AW_CUDA_TRY(cudaSetDevice(dev));
    return AW_OK;
}

struct ReprojArgs {
    const float *src;
    float *dst;
    double R[9];                 // source (l', m', n') = R (l, m, n) of the destination
    float Rf[9];                 // R in FP32, for the cheap outside test
    double dl_d, cx_d, cy_d;     // destination frame
    double inv_dl_s, cx_s, cy_s; // source frame
    int Nd, Ns, nplane;
    float fill;
};

// Keys cubic convolution (a = -1/2) weights of the samples at -1, 0, 1, 2
// from floor(x), t = x - floor(x) in [0, 1): FP32 (the position and its floor
// are FP64).
__device__ __forceinline__ void keys4(float t, float w[4]) {
    const float a = -0.5f;
    const float s[4] = {1.0f + t, t, 1.0f - t, 2.0f - t};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float x = s[i];
        w[i] = (x <= 1.0f) ? (((a + 2.0f) * x - (a + 3.0f)) * x * x + 1.0f)
                           : (((a * x - 5.0f * a) * x + 8.0f * a) * x - 4.0f * a);
    }
}

template <int INTERP>
__global__ void reproject_kernel(ReprojArgs a) {
    constexpr int K = (INTERP == AW_INTERP_CUBIC) ? 4 : 2;
    constexpr int O = (INTERP == AW_INTERP_CUBIC) ? -1 : 0;
    const int64_t npix = (int64_t)a.Nd * a.Nd;
    const int64_t splane = (int64_t)a.Ns * a.Ns;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int qy = (int)(i / a.Nd), qx = (int)(i % a.Nd);
        {
            // FP32 first: its position error is below 0.01 pixel for any frame pair on the
            // sphere, so a position more than 1.5 pixels outside the source's stencil range
            // is outside in FP64 too
            const float lf = ((float)qx - (float)a.cx_d) * (float)a.dl_d;
            const float mf = ((float)qy - (float)a.cy_d) * (float)a.dl_d;
            const float nf = sqrtf(fmaxf(1.0f - lf * lf - mf * mf, 0.0f));
            const float xf = (a.Rf[0] * lf + a.Rf[1] * mf + a.Rf[2] * nf) * (float)a.inv_dl_s + (float)a.cx_s;
            const float yf = (a.Rf[3] * lf + a.Rf[4] * mf + a.Rf[5] * nf) * (float)a.inv_dl_s + (float)a.cy_s;
            const float lo = (float)(-O) - 1.5f, hi = (float)(a.Ns - K - O) + 2.5f;
            if (!(xf >= lo && xf <= hi && yf >= lo && yf <= hi)) {
                for (int p = 0; p < a.nplane; ++p) a.dst[p * npix + i] = a.fill;
                continue;
            }
        }
        const double l = ((double)qx - a.cx_d) * a.dl_d;
        const double m = ((double)qy - a.cy_d) * a.dl_d;
        const double r2 = l * l + m * m;
        bool ok = r2 <= 1.0;
        const double n = ok ? sqrt(1.0 - r2) : 0.0;
        const double ls = a.R[0] * l + a.R[1] * m + a.R[2] * n;
        const double ms = a.R[3] * l + a.R[4] * m + a.R[5] * n;
        const double ns = a.R[6] * l + a.R[7] * m + a.R[8] * n;
        ok = ok && ns > 0.0;
        const double x = ls * a.inv_dl_s + a.cx_s;
        const double y = ms * a.inv_dl_s + a.cy_s;
        const double fx = floor(x), fy = floor(y);
        // stencil inside the source image (compared in FP64 before any int conversion)
        ok = ok && fx + O >= 0.0 && fx + O + K - 1 <= (double)(a.Ns - 1) && fy + O >= 0.0 &&
             fy + O + K - 1 <= (double)(a.Ns - 1);
        if (!ok) {
            for (int p = 0; p < a.nplane; ++p) a.dst[p * npix + i] = a.fill;
            continue;
        }
        const int x0 = (int)fx + O, y0 = (int)fy + O;
        float wx[K], wy[K];
        const float tx = (float)(x - fx), ty = (float)(y - fy);
        if constexpr (INTERP == AW_INTERP_CUBIC) {
            keys4(tx, wx);
            keys4(ty, wy);
        } else {
            wx[0] = 1.0f - tx;
            wx[1] = tx;
            wy[0] = 1.0f - ty;
            wy[1] = ty;
        }
        for (int p = 0; p < a.nplane; ++p) {
            const float *s = a.src + p * splane + (int64_t)y0 * a.Ns + x0;
            float acc = 0.f;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                float row = 0.f;
#pragma unroll
                for (int c = 0; c < K; ++c) row = fmaf(wx[c], __ldg(s + (int64_t)r * a.Ns + c), row);
                acc = fmaf(wy[r], row, acc);
            }
            a.dst[p * npix + i] = acc;
        }
    }
}

__global__ void combine_kernel(const float *images, const float *beams, const float *gamma, int nfield, int nplane,
                               int64_t npix, float *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float g = gamma[i];
        for (int p = 0; p < nplane; ++p) {
            float s = 0.f;
            for (int f = 0; f < nfield; ++f)
                s = fmaf(beams[f * npix + i], images[((int64_t)f * nplane + p) * npix + i], s);
            out[p * npix + i] = g * s;
        }
    }
}

// uvw' = R uvw per row (FP64)
__global__ void rotate_uvw_kernel(const double *uvw, double *out, int64_t nrow, double r0, double r1, double r2,
                                  double r3, double r4, double r5, double r6, double r7, double r8) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrow; i += (int64_t)gridDim.x * blockDim.x) {
        const double u = uvw[3 * i], v = uvw[3 * i + 1], w = uvw[3 * i + 2];
        out[3 * i] = r0 * u + r1 * v + r2 * w;
        out[3 * i + 1] = r3 * u + r4 * v + r5 * w;
        out[3 * i + 2] = r6 * u + r7 * v + r8 * w;
    }
}

// V' = V exp(2 pi i (w' - w) nu / c), the phase in FP64
__global__ void rotate_vis_kernel(const double *uvw, const uint32_t *row, const uint16_t *chan, const double *freq,
                                  int64_t nvis, int npol, const float2 *vin, float2 *vout, double r6, double r7,
                                  double r8) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvis; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = row[i];
        const double u = uvw[3 * r], v = uvw[3 * r + 1], w = uvw[3 * r + 2];
        const double dw = (r6 * u + r7 * v + r8 * w) - w;
        double sp, cp;
        sincos(2.0 * M_PI * (dw * (freq[chan[i]] / AW_C_LIGHT)), &sp, &cp);
        const float c = (float)cp, sn = (float)sp;
        for (int k = 0; k < npol; ++k) {
            const float2 a = vin[i * npol + k];
            vout[i * npol + k] = make_float2(a.x * c - a.y * sn, a.x * sn + a.y * c);
        }
    }
}

int nblk(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

// Orthonormal axes (east, north, centre) of the tangent frame at (ra0, dec0)
// as the rows of B: (l, m, n) = B s for a unit sky vector s.
void frame_axes(double ra0, double dec0, double B[9]) {
    const double sa = std::sin(ra0), ca = std::cos(ra0), sd = std::sin(dec0), cd = std::cos(dec0);
    const double b[9] = {-sa, ca, 0.0, -sd * ca, -sd * sa, cd, cd * ca, cd * sa, sd};
    for (int i = 0; i < 9; ++i) B[i] = b[i];
}

int check_frame(const aw_sky_frame *f, const char *name) {
    if (!f) return aw_set_error(AW_EINVAL, "%s frame is NULL", name);
    if (f->N < 4 || !(f->dl > 0.0) || !std::isfinite(f->dl) || !std::isfinite(f->cx) || !std::isfinite(f->cy) ||
        !std::isfinite(f->ra0) || !std::isfinite(f->dec0))
        return aw_set_error(AW_EINVAL, "%s frame: N=%d dl=%g", name, f->N, f->dl);
    return AW_OK;
}

#define MO_GUARD_BEGIN \
    AW_TRACE();         \
    try {
#define MO_GUARD_END                                                   \
    }                                                                  \
    catch (const std::bad_alloc &) {                                   \
        return aw_set_error(AW_ENOMEM, "host allocation failed");      \
    }                                                                  \
    catch (...) {                                                      \
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");    \
    }

}  // namespace

extern "C" {

int aw_reproject(aw_ctx *ctx, const float *src, const aw_sky_frame *sf, float *dst, const aw_sky_frame *df,
                 int32_t nplane, int32_t interp, float fill, void *stream) {
    MO_GUARD_BEGIN
    if (!ctx || !src || !dst) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = check_frame(sf, "source");
    if (rc) return rc;
    rc = check_frame(df, "destination");
    if (rc) return rc;
    if (nplane < 1) return aw_set_error(AW_EINVAL, "nplane %d", nplane);
    if (interp != AW_INTERP_BILINEAR && interp != AW_INTERP_CUBIC) return aw_set_error(AW_EINVAL, "interp %d", interp);
    rc = use_device(ctx->device);
    if (rc) return rc;
    ReprojArgs a;
    double Bs[9], Bd[9];
    frame_axes(sf->ra0, sf->dec0, Bs);
    frame_axes(df->ra0, df->dec0, Bd);
    // s = Bd^T (l, m, n)_d  ->  (l, m, n)_s = Bs s = (Bs Bd^T) (l, m, n)_d
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += Bs[3 * i + k] * Bd[3 * j + k];
            a.R[3 * i + j] = v;
            a.Rf[3 * i + j] = (float)v;
        }
    a.src = src;
    a.dst = dst;
    a.dl_d = df->dl;
    a.cx_d = df->cx;
    a.cy_d = df->cy;
    a.inv_dl_s = 1.0 / sf->dl;
    a.cx_s = sf->cx;
    a.cy_s = sf->cy;
    a.Nd = df->N;
    a.Ns = sf->N;
    a.nplane = nplane;
    a.fill = fill;
    const int64_t npix = (int64_t)df->N * df->N;
    cudaStream_t s = S_(stream);
    if (interp == AW_INTERP_CUBIC)
        reproject_kernel<AW_INTERP_CUBIC><<<nblk(npix, 256), 256, 0, s>>>(a);
    else
        reproject_kernel<AW_INTERP_BILINEAR><<<nblk(npix, 256), 256, 0, s>>>(a);
    AW_CHECK_LAUNCH();
    return AW_OK;
    MO_GUARD_END
}

int aw_phase_rotate(aw_ctx *ctx, const aw_vis_desc *vd, double *uvw_out, const void *vis, void *vis_out, int32_t npol,
                    double ra_from, double dec_from, double ra_to, double dec_to, void *stream) {
    MO_GUARD_BEGIN
    if (!ctx || !vd) return aw_set_error(AW_EINVAL, "NULL argument");
    if (npol != 1 && npol != 4) return aw_set_error(AW_EINVAL, "npol %d", npol);
    if (vd->nvis < 0 || vd->nrow < 0) return aw_set_error(AW_EINVAL, "negative sizes");
    if (vd->nvis > 0 && (!vd->uvw || !vd->row_of_vis || !vd->chan_of_vis || !vd->freq || !vis || !vis_out))
        return aw_set_error(AW_EINVAL, "vis descriptor or buffers incomplete");
    if (uvw_out && uvw_out == vd->uvw) return aw_set_error(AW_EINVAL, "uvw_out must not alias the input uvw");
    if (!std::isfinite(ra_from) || !std::isfinite(dec_from) || !std::isfinite(ra_to) || !std::isfinite(dec_to))
        return aw_set_error(AW_EINVAL, "phase centres must be finite");
    int rc = use_device(ctx->device);
    if (rc) return rc;
    double Bf[9], Bt[9], R[9];
    frame_axes(ra_from, dec_from, Bf);
    frame_axes(ra_to, dec_to, Bt);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += Bt[3 * i + k] * Bf[3 * j + k];
            R[3 * i + j] = v;
        }
    cudaStream_t s = S_(stream);
    if (vd->nvis > 0) {
        rotate_vis_kernel<<<nblk(vd->nvis, 256), 256, 0, s>>>(vd->uvw, vd->row_of_vis, vd->chan_of_vis, vd->freq,
                                                             vd->nvis, npol, reinterpret_cast<const float2 *>(vis),
                                                             reinterpret_cast<float2 *>(vis_out), R[6], R[7], R[8]);
        AW_CHECK_LAUNCH();
    }
    if (uvw_out && vd->nrow > 0) {
        rotate_uvw_kernel<<<nblk(vd->nrow, 256), 256, 0, s>>>(vd->uvw, uvw_out, vd->nrow, R[0], R[1], R[2], R[3], R[4],
                                                             R[5], R[6], R[7], R[8]);
        AW_CHECK_LAUNCH();
    }
    return AW_OK;
    MO_GUARD_END
}

int aw_mosaic_combine(aw_ctx *ctx, const float *images, const float *beams, const float *gamma, int32_t nfield,
                      int32_t nplane, int32_t N, float *out, void *stream) {
    MO_GUARD_BEGIN
    if (!ctx || !images || !beams || !gamma || !out) return aw_set_error(AW_EINVAL, "NULL argument");
    if (nfield < 1 || nplane < 1 || N < 1) return aw_set_error(AW_EINVAL, "nfield=%d nplane=%d N=%d", nfield, nplane, N);
    int rc = use_device(ctx->device);
    if (rc) return rc;
    const int64_t npix = (int64_t)N * N;
    combine_kernel<<<nblk(npix, 256), 256, 0, S_(stream)>>>(images, beams, gamma, nfield, nplane, npix, out);
    AW_CHECK_LAUNCH();
    return AW_OK;
    MO_GUARD_END
}

}  // extern "C"
