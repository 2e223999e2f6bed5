// uv grid -> dirty image (Sec. 2.2: FFTs on the GPU) and the mosaic
// weighting gamma(l, m) of Eq. 1 (Sec. 2.2).
#include <cmath>

#include "aw_internal.h"

namespace {

// (-1)^(x + y) moves the DC cell N/2 to 0 and back (N a multiple of 4).
__global__ void checker_kernel(float2 *g, int N, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = i % ((int64_t)N * N);
        const int y = (int)(pix / N), x = (int)(pix % N);
        if ((x + y) & 1) {
            float2 v = g[i];
            g[i] = make_float2(-v.x, -v.y);
        }
    }
}

// image = (-1)^(qx+qy) Re(Z) / (c[qx] c[qy]) / weight_sum, zero on row/col 0
__global__ void gridcorr_kernel(const float2 *Z, const float *corr, int N, int64_t total,
                                float inv_wsum, float *img) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = i % ((int64_t)N * N);
        const int y = (int)(pix / N), x = (int)(pix % N);
        float v = 0.f;
        if (x != 0 && y != 0) {
            const float re = ((x + y) & 1) ? -Z[i].x : Z[i].x;
            v = re / (corr[x] * corr[y]) * inv_wsum;
        }
        img[i] = v;
    }
}

// grid = (-1)^(qx+qy) I(q) / (c[qx] c[qy]) as complex, zero on row/col 0 (the
// first half of the model-image -> grid step; a forward FFT and the checker follow)
__global__ void image_prep_kernel(const float *img, const float *corr, int N, int64_t total, float2 *g) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pix = i % ((int64_t)N * N);
        const int y = (int)(pix / N), x = (int)(pix % N);
        float v = 0.f;
        if (x != 0 && y != 0) {
            v = img[i] / (corr[x] * corr[y]);
            if ((x + y) & 1) v = -v;
        }
        g[i] = make_float2(v, 0.f);
    }
}

__global__ void gamma_max_kernel(const float *B, int nfield, int64_t npix, unsigned int *maxbits) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int f = 0; f < nfield; ++f) {
            const float b = B[(int64_t)f * npix + i];
            s = fmaf(b, b, s);
        }
        m = fmaxf(m, sqrtf(s));
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(m));
}

__global__ void gamma_apply_kernel(const float *B, int nfield, int64_t npix, const unsigned int *maxbits,
                                   float eps, float *gamma) {
    const float mx = __uint_as_float(*maxbits);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int f = 0; f < nfield; ++f) {
            const float b = B[(int64_t)f * npix + i];
            s = fmaf(b, b, s);
        }
        const float pbp = (mx > 0.f) ? sqrtf(s) / mx : 0.f;   // [sqrt(sum B^2) / max]_pbp
        const float wc = (s > 0.f) ? 1.0f / s : 0.f;           // [1 / sum B^2]_wc
        gamma[i] = (pbp < eps || s == 0.f) ? 0.f : pbp * wc;
    }
}

int nblocks(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

int aw_ctx_gridcorr(aw_ctx *ctx, int N, double W, float **out) {
    auto key = std::make_pair(N, W);
    auto it = ctx->gridcorr.find(key);
    if (it != ctx->gridcorr.end()) { *out = it->second; return AW_OK; }
    const aw_pswf p = aw_pswf_make(M_PI * W / 2.0);
    std::vector<float> c(N);
    for (int q = 0; q < N; ++q) c[q] = (q == 0) ? 0.f : (float)p.eval((q - N / 2) * 2.0 / N);
    float *d = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&d, sizeof(float) * N));
    AW_CUDA_TRY(cudaMemcpy(d, c.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
    ctx->gridcorr[key] = d;
    *out = d;
    return AW_OK;
}

int aw_fft_to_image_impl(aw_ctx *ctx, int N, int npol, double W, void *grid, double weight_sum,
                         float *image, cudaStream_t s) {
    if (N % 4) return aw_set_error(AW_EINVAL, "N must be a multiple of 4");
    if (!(weight_sum > 0)) return aw_set_error(AW_EINVAL, "weight_sum must be positive");
    float *corr = nullptr;
    int rc = aw_ctx_gridcorr(ctx, N, W, &corr);
    if (rc) return rc;
    cufftHandle plan;
    rc = aw_ctx_fft_plan(ctx, 2, N, npol, CUFFT_C2C, &plan);
    if (rc) return rc;
    AW_CUFFT_TRY(cufftSetStream(plan, s));
    const int64_t total = (int64_t)npol * N * N;
    float2 *g = reinterpret_cast<float2 *>(grid);
    checker_kernel<<<nblocks(total, 256), 256, 0, s>>>(g, N, total);
    AW_CHECK_LAUNCH();
    AW_CUFFT_TRY(cufftExecC2C(plan, reinterpret_cast<cufftComplex *>(g), reinterpret_cast<cufftComplex *>(g),
                              CUFFT_INVERSE));
    gridcorr_kernel<<<nblocks(total, 256), 256, 0, s>>>(g, corr, N, total, (float)(1.0 / weight_sum), image);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

// G(g) = sum_q I(q) / c(q) exp(-2 pi i (g - N/2)(q - N/2) / N): with N a multiple
// of 4 the centring phases reduce to (-1)^(q) before and (-1)^(g) after a plain
// forward FFT.
int aw_image_to_grid_impl(aw_ctx *ctx, int N, int npol, double W, const float *image, void *grid,
                          cudaStream_t s) {
    if (N % 4) return aw_set_error(AW_EINVAL, "N must be a multiple of 4");
    float *corr = nullptr;
    int rc = aw_ctx_gridcorr(ctx, N, W, &corr);
    if (rc) return rc;
    cufftHandle plan;
    rc = aw_ctx_fft_plan(ctx, 2, N, npol, CUFFT_C2C, &plan);
    if (rc) return rc;
    AW_CUFFT_TRY(cufftSetStream(plan, s));
    const int64_t total = (int64_t)npol * N * N;
    float2 *g = reinterpret_cast<float2 *>(grid);
    image_prep_kernel<<<nblocks(total, 256), 256, 0, s>>>(image, corr, N, total, g);
    AW_CHECK_LAUNCH();
    AW_CUFFT_TRY(cufftExecC2C(plan, reinterpret_cast<cufftComplex *>(g), reinterpret_cast<cufftComplex *>(g),
                              CUFFT_FORWARD));
    checker_kernel<<<nblocks(total, 256), 256, 0, s>>>(g, N, total);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

int aw_mosaic_gamma_impl(aw_ctx *ctx, const float *beams, int nfield, int N, float eps, float *gamma,
                         cudaStream_t s) {
    const int64_t npix = (int64_t)N * N;
    AW_CUDA_TRY(cudaMemsetAsync(ctx->d_scratch, 0, sizeof(unsigned int), s));
    gamma_max_kernel<<<nblocks(npix, 256), 256, 0, s>>>(beams, nfield, npix, ctx->d_scratch);
    AW_CHECK_LAUNCH();
    gamma_apply_kernel<<<nblocks(npix, 256), 256, 0, s>>>(beams, nfield, npix, ctx->d_scratch, eps, gamma);
    AW_CHECK_LAUNCH();
    return AW_OK;
}
