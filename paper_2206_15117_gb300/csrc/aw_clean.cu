// Cleaning: Cotton-Schwab major cycles around a Hogbom minor cycle.
//
// arXiv:2206.15117 Sec. 2.1: the imager cleans with the Cotton-Schwab
// algorithm (number of clean cycles, loop gain, cycle factor, threshold);
// Sec. 4 names Hogbom cleaning as its iterative, hard-to-parallelise part.
// The readings the paper leaves open are stated with the declarations in
// aw.h.  Major-cycle transforms reuse the gridding, image and degridding
// paths; the minor cycle runs in one CTA with per-tile maxima so that each
// iteration rescans only the tiles its subtraction touched.
#include <algorithm>
#include <cmath>
#include <cstring>
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

int nblk(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// ctx->d_scratch words used here
constexpr int SCR_R0 = 4;        // main-lobe radius
constexpr int SCR_SIDE = 5;      // sidelobe level (float bits, >= 0)
constexpr int SCR_PEAK = 6;      // window peak |I| (float bits, >= 0)
constexpr int SCR_NITER = 7;     // Hogbom iterations
constexpr int SCR_BAR_COUNT = 8; // grid barrier: arrivals
constexpr int SCR_BAR_GEN = 9;   // grid barrier: generation
constexpr int SCR_BAR_ERR = 10;  // grid barrier: set when a wait gave up
// spin limit of one barrier wait: 2^24 polls with a 64 ns back-off, about 9 s on GB300
constexpr long long BAR_SPIN_LIMIT = 1ll << 24;

// ---------------------------------------------------------------- sidelobe
// r0 = first x > 0 with psf[c][c + x] <= 0 (N/2 if none), one warp.
__global__ void psf_r0_kernel(const float *psf, int N, unsigned int *scr) {
    const int c = N / 2, lane = threadIdx.x;
    int r0 = N / 2;
    for (int base = 1; base < N - c; base += 32) {
        const int x = base + lane;
        const bool hit = x < N - c && psf[(int64_t)c * N + c + x] <= 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) { r0 = base + __ffs(m) - 1; break; }
    }
    if (lane == 0) scr[SCR_R0] = (unsigned)r0;
}

__global__ void psf_side_kernel(const float *psf, int N, unsigned int *scr) {
    const int c = N / 2;
    const int64_t r0 = scr[SCR_R0];
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)N * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dy = i / N - c, dx = i % N - c;
        const int64_t q = N / 4;
        if (dx * dx + dy * dy > r0 * r0 && dx < q && -dx < q && dy < q && -dy < q) m = fmaxf(m, fabsf(psf[i]));
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&scr[SCR_SIDE], __float_as_uint(m));
}

// ---------------------------------------------------------------- window peak
__global__ void window_peak_kernel(const float *img, int N, int x0, int y0, int x1, int y1, unsigned int *scr) {
    const int w = x1 - x0;
    const int64_t cnt = (int64_t)w * (y1 - y0);
    float m = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(img[(int64_t)(y0 + e / w) * N + x0 + e % w]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&scr[SCR_PEAK], __float_as_uint(m));
}

// ---------------------------------------------------------------- Hogbom
// |I| and the pixel index packed so that the unsigned maximum is the largest
// |I| with the lowest index; 0 means "no pixel".
__device__ __forceinline__ unsigned long long hb_pack(float v, uint32_t idx) {
    return ((unsigned long long)__float_as_uint(fabsf(v)) << 32) | (unsigned long long)(0xFFFFFFFFu - idx);
}

struct HbGeom {
    int N, T, TX;
    int x0, y0, x1, y1;
};

// Block-wide maximum (all threads call; result valid in every thread).
__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long *red) {
    for (int o = 16; o; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? red[lane] : 0ull;
        for (int o = 16; o; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
            v = u > v ? u : v;
        }
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    return red[32];
}

// Maximum of tile t over its window pixels, by the whole block.
__device__ unsigned long long tile_scan(const float *R0, const HbGeom &g, int t, unsigned long long *red) {
    const int tx = t % g.TX, ty = t / g.TX;
    const int xa = max(tx * g.T, g.x0), xb = min((tx + 1) * g.T, g.x1);
    const int ya = max(ty * g.T, g.y0), yb = min((ty + 1) * g.T, g.y1);
    unsigned long long v = 0ull;
    if (xa < xb && ya < yb) {
        const int w = xb - xa, cnt = w * (yb - ya);
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const uint32_t idx = (uint32_t)(ya + e / w) * (uint32_t)g.N + (uint32_t)(xa + e % w);
            const unsigned long long p = hb_pack(R0[idx], idx);
            v = p > v ? p : v;
        }
    }
    return block_max_u64(v, red);
}

__global__ void hb_tiles_kernel(const float *R0, HbGeom g, unsigned long long *tmax) {
    __shared__ unsigned long long red[33];
    const unsigned long long v = tile_scan(R0, g, blockIdx.x, red);
    if (threadIdx.x == 0) tmax[blockIdx.x] = v;
}

constexpr int HB_THREADS = 256;

// Barrier over all blocks of a cooperative launch (co-residency guaranteed by
// the launch).  The last block to arrive resets the count and advances the
// generation; the others poll the generation with a bounded wait.  A wait that
// runs out sets the error word and returns false, so that no block can wait
// for ever; the caller then leaves its loop.
__device__ bool grid_barrier(unsigned int *scr, unsigned int nblocks, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = scr + SCR_BAR_GEN;
        const unsigned int g0 = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(scr + SCR_BAR_COUNT, 1u) + 1u;
        int ok = 1;
        if (arrived == nblocks) {
            atomicExch(scr + SCR_BAR_COUNT, 0u);
            __threadfence();
            atomicAdd(scr + SCR_BAR_GEN, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                if (++spins > BAR_SPIN_LIMIT || *(volatile unsigned int *)(scr + SCR_BAR_ERR)) {
                    atomicExch(scr + SCR_BAR_ERR, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Self-test of the barrier's bounded wait: one block that expects a second
// arrival which never comes (the arrival count is never reached).
__global__ void barrier_timeout_kernel(unsigned int *scr) {
    __shared__ int s_ok;
    grid_barrier(scr, 2u, &s_ok);
}

// Maximum of tile t over its window pixels, by one block, reading the
// residual through L2 (other blocks write it between grid barriers).
__device__ unsigned long long tile_scan_l2(const float *R0, const HbGeom &g, int t, unsigned long long *red) {
    const int tx = t % g.TX, ty = t / g.TX;
    const int xa = max(tx * g.T, g.x0), xb = min((tx + 1) * g.T, g.x1);
    const int ya = max(ty * g.T, g.y0), yb = min((ty + 1) * g.T, g.y1);
    unsigned long long v = 0ull;
    if (xa < xb && ya < yb) {
        const int w = xb - xa, cnt = w * (yb - ya);
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const uint32_t idx = (uint32_t)(ya + e / w) * (uint32_t)g.N + (uint32_t)(xa + e % w);
            const unsigned long long p = hb_pack(__ldcg(R0 + idx), idx);
            v = p > v ? p : v;
        }
    }
    return block_max_u64(v, red);
}

// The minor cycle as one cooperative grid.  Per iteration: every block finds
// the same peak from the tile maxima (global, read through L2) and the same
// component (gain x residual, all planes); after a grid barrier block 0 adds
// the component to the model and all blocks subtract component x psf over the
// patch (FP32, one rounding per multiply and per subtraction); after a second
// barrier the blocks rescan the touched tiles; a third barrier ends the
// iteration.  Every block takes the same stop decision from the same data.
__global__ void __launch_bounds__(HB_THREADS) hogbom_kernel(float *R, const float *psf, float *model, int npol,
                                                            HbGeom g, float gain, float thr, int max_iter,
                                                            int h, unsigned long long *tmax, unsigned int *scr) {
    __shared__ int s_ok;
    __shared__ unsigned long long red[33];
    __shared__ float comp[4];
    __shared__ int s_stop, s_py, s_px;
    __shared__ uint32_t s_idx;
    const int ntiles = g.TX * g.TX;
    const int64_t NN = (int64_t)g.N * g.N;
    const int c = g.N / 2;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int n = 0;; ++n) {
        unsigned long long v = 0ull;
        for (int i = threadIdx.x; i < ntiles; i += blockDim.x) {
            const unsigned long long t = __ldcg(tmax + i);
            v = t > v ? t : v;
        }
        const unsigned long long best = block_max_u64(v, red);
        if (threadIdx.x == 0) {
            int stop = (best == 0ull || n >= max_iter) ? 1 : 0;
            if (!stop) {
                const uint32_t idx = 0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFull);
                if (fabsf(__ldcg(R + idx)) < thr) {
                    stop = 1;
                } else {
                    for (int s = 0; s < npol; ++s) comp[s] = __fmul_rn(gain, __ldcg(R + s * NN + idx));
                    s_idx = idx;
                    s_py = (int)(idx / (uint32_t)g.N);
                    s_px = (int)(idx % (uint32_t)g.N);
                }
            }
            s_stop = stop;
            if (stop && blockIdx.x == 0) scr[SCR_NITER] = (unsigned)n;
        }
        __syncthreads();
        if (s_stop) break;
        if (!grid_barrier(scr, gridDim.x, &s_ok)) break;  // every block has read the residual at the peak
        if (blockIdx.x == 0 && threadIdx.x < npol) {
            const int64_t o = threadIdx.x * NN + s_idx;
            model[o] = __fadd_rn(model[o], comp[threadIdx.x]);
        }
        const int py = s_py, px = s_px;
        const int ya = max(0, py - h), yb = min(g.N, py + h + 1);
        const int xa = max(0, px - h), xb = min(g.N, px + h + 1);
        const int w = xb - xa;
        const int64_t cnt = (int64_t)w * (yb - ya);
        for (int64_t e = gtid; e < npol * cnt; e += gthreads) {
            const int s = (int)(e / cnt);
            const int64_t r = e - s * cnt;
            const int y = ya + (int)(r / w), x = xa + (int)(r % w);
            float *p = R + s * NN + (int64_t)y * g.N + x;
            *p = __fsub_rn(__ldcg(p), __fmul_rn(comp[s], psf[(int64_t)(c + y - py) * g.N + (c + x - px)]));
        }
        if (!grid_barrier(scr, gridDim.x, &s_ok)) break;  // the patch is subtracted everywhere
        const int rxa = max(xa, g.x0), rxb = min(xb, g.x1), rya = max(ya, g.y0), ryb = min(yb, g.y1);
        if (rxa < rxb && rya < ryb) {
            const int tx0 = rxa / g.T, tx1 = (rxb - 1) / g.T, ty0 = rya / g.T, ty1 = (ryb - 1) / g.T;
            const int ntx = tx1 - tx0 + 1, nt = ntx * (ty1 - ty0 + 1);
            for (int k = blockIdx.x; k < nt; k += gridDim.x) {
                const int t = (ty0 + k / ntx) * g.TX + tx0 + k % ntx;
                const unsigned long long tv = tile_scan_l2(R, g, t, red);
                if (threadIdx.x == 0) tmax[t] = tv;
            }
        }
        if (!grid_barrier(scr, gridDim.x, &s_ok)) break;  // the tile maxima are current
    }
}

// ---------------------------------------------------------------- clean helpers
__global__ void unit_vis_kernel(float2 *v, int64_t nvis, int npol) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvis * npol;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % npol);
        v[i] = make_float2((c == 0 || c == 3) ? 1.f : 0.f, 0.f);
    }
}

__global__ void psf_norm_kernel(const float *plane0, int N, float *psf) {
    const float p0 = plane0[(int64_t)(N / 2) * N + N / 2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)N * N;
         i += (int64_t)gridDim.x * blockDim.x)
        psf[i] = plane0[i] / p0;
}

int check_window(const int32_t *win, int N) {
    if (!win) return aw_set_error(AW_EINVAL, "window is NULL");
    if (win[0] < 0 || win[1] < 0 || win[2] > N || win[3] > N || win[0] >= win[2] || win[1] >= win[3])
        return aw_set_error(AW_EINVAL, "window (%d, %d, %d, %d) not a non-empty box inside the %d^2 image",
                            win[0], win[1], win[2], win[3], N);
    return AW_OK;
}

HbGeom geom_of(int N, const int32_t *win) {
    HbGeom g;
    g.N = N;
    g.T = std::max(64, (N + 63) / 64);
    g.TX = (N + g.T - 1) / g.T;
    g.x0 = win[0];
    g.y0 = win[1];
    g.x1 = win[2];
    g.y1 = win[3];
    return g;
}

// Run barrier_timeout_kernel: AW_ETIMEOUT once the wait has given up.
int barrier_selftest_impl(aw_ctx *ctx, cudaStream_t s) {
    AW_CUDA_TRY(cudaMemsetAsync(ctx->d_scratch + SCR_BAR_COUNT, 0, 3 * sizeof(unsigned int), s));
    barrier_timeout_kernel<<<1, 32, 0, s>>>(ctx->d_scratch);
    AW_CHECK_LAUNCH();
    unsigned int w = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&w, ctx->d_scratch + SCR_BAR_ERR, sizeof(w), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    AW_CUDA_TRY(cudaMemsetAsync(ctx->d_scratch + SCR_BAR_COUNT, 0, 3 * sizeof(unsigned int), s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    return w ? aw_set_error(AW_ETIMEOUT, "grid barrier wait gave up") : AW_OK;
}

int hogbom_impl(aw_ctx *ctx, float *R, const float *psf, int npol, int N, float gain, float thr, int max_iter,
                int h, const int32_t *win, float *model, int32_t *n_iter, cudaStream_t s) {
    HbGeom g = geom_of(N, win);
    const int ntiles = g.TX * g.TX;
    unsigned long long *tmax = nullptr;
    AW_CUDA_TRY(cudaMallocAsync(&tmax, sizeof(unsigned long long) * ntiles, s));
    hb_tiles_kernel<<<ntiles, 256, 0, s>>>(R, g, tmax);
    cudaError_t e = cudaGetLastError();
    // one co-resident block per SM (at most 2): the barriers cost more than the work
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hogbom_kernel, HB_THREADS, 0);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorCooperativeLaunchTooLarge;
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_scratch + SCR_BAR_COUNT, 0, 3 * sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        const int blocks = ctx->sm_count * std::min(per_sm, 2);
        void *args[] = {&R, (void *)&psf, &model, &npol, &g, &gain, &thr, &max_iter, &h, &tmax, &ctx->d_scratch};
        e = cudaLaunchCooperativeKernel((const void *)hogbom_kernel, dim3(blocks), dim3(HB_THREADS), args, 0, s);
    }
    cudaFreeAsync(tmax, s);
    if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "hogbom: %s", cudaGetErrorString(e));
    unsigned int w[4] = {0, 0, 0, 0};  // iterations, barrier count, generation, error
    AW_CUDA_TRY(cudaMemcpyAsync(w, ctx->d_scratch + SCR_NITER, sizeof(w), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    if (w[3]) return aw_set_error(AW_ETIMEOUT, "hogbom: a grid barrier wait gave up; results are invalid");
    *n_iter = (int32_t)w[0];
    return AW_OK;
}

int sidelobe_impl(aw_ctx *ctx, const float *psf, int N, float *out, cudaStream_t s) {
    AW_CUDA_TRY(cudaMemsetAsync(ctx->d_scratch + SCR_SIDE, 0, sizeof(unsigned int), s));
    psf_r0_kernel<<<1, 32, 0, s>>>(psf, N, ctx->d_scratch);
    AW_CHECK_LAUNCH();
    psf_side_kernel<<<nblk((int64_t)N * N, 256), 256, 0, s>>>(psf, N, ctx->d_scratch);
    AW_CHECK_LAUNCH();
    unsigned int bits = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&bits, ctx->d_scratch + SCR_SIDE, sizeof(bits), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(out, &bits, sizeof(float));
    return AW_OK;
}

int window_peak_impl(aw_ctx *ctx, const float *img, int N, const int32_t *win, float *out, cudaStream_t s) {
    AW_CUDA_TRY(cudaMemsetAsync(ctx->d_scratch + SCR_PEAK, 0, sizeof(unsigned int), s));
    const int64_t cnt = (int64_t)(win[2] - win[0]) * (win[3] - win[1]);
    window_peak_kernel<<<nblk(cnt, 256), 256, 0, s>>>(img, N, win[0], win[1], win[2], win[3], ctx->d_scratch);
    AW_CHECK_LAUNCH();
    unsigned int bits = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&bits, ctx->d_scratch + SCR_PEAK, sizeof(bits), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(out, &bits, sizeof(float));
    return AW_OK;
}

struct DevMem {
    void *p = nullptr;
    ~DevMem() { if (p) aw_dev_free(p); }
};

int check_plan_kset(const aw_plan *p, const aw_kernel_set *k) {
    if (!p || !k) return aw_set_error(AW_EINVAL, "plan/kset is NULL");
    if (p->N != k->spec.N || p->OS != k->spec.OS || p->npol != k->spec.npol || p->nbins != k->nbins || p->ntype != k->ntype ||
        p->bin_support != k->bin_support)
        return aw_set_error(AW_EINVAL, "kernel set geometry does not match the plan");
    return AW_OK;
}

#define CL_GUARD_BEGIN \
    AW_TRACE();         \
    try {
#define CL_GUARD_END                                                   \
    }                                                                  \
    catch (const std::bad_alloc &) {                                   \
        return aw_set_error(AW_ENOMEM, "host allocation failed");      \
    }                                                                  \
    catch (...) {                                                      \
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");    \
    }

}  // namespace

int aw_barrier_selftest(aw_ctx *ctx, cudaStream_t s) { return barrier_selftest_impl(ctx, s); }

extern "C" {

int aw_image_to_grid(aw_ctx *ctx, const aw_kernel_set *k, const float *image, void *grid, void *stream) {
    CL_GUARD_BEGIN
    if (!ctx || !k || !image || !grid) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = use_device(ctx->device);
    if (rc) return rc;
    return aw_image_to_grid_impl(ctx, k->spec.N, k->spec.npol, k->spec.W, image, grid, S_(stream));
    CL_GUARD_END
}

int aw_degrid_subtract(aw_ctx *ctx, const aw_plan *p, const aw_kernel_set *k, const void *grid, const void *vis,
                       void *vis_out, void *stream) {
    CL_GUARD_BEGIN
    if (!ctx) return aw_set_error(AW_EINVAL, "ctx is NULL");
    int rc = check_plan_kset(p, k);
    if (rc) return rc;
    if (!grid || ((!vis || !vis_out) && p->nvis)) return aw_set_error(AW_EINVAL, "grid/vis/vis_out is NULL");
    rc = use_device(ctx->device);
    if (rc) return rc;
    return aw_launch_degrid(p, k, grid, vis_out, S_(stream), vis);
    CL_GUARD_END
}

int aw_psf_sidelobe(aw_ctx *ctx, const float *psf, int32_t N, float *sidelobe, void *stream) {
    CL_GUARD_BEGIN
    if (!ctx || !psf || !sidelobe) return aw_set_error(AW_EINVAL, "NULL argument");
    if (N < 2) return aw_set_error(AW_EINVAL, "N=%d", N);
    int rc = use_device(ctx->device);
    if (rc) return rc;
    return sidelobe_impl(ctx, psf, N, sidelobe, S_(stream));
    CL_GUARD_END
}

int aw_hogbom(aw_ctx *ctx, float *residual, const float *psf, int32_t npol, int32_t N, float gain,
              float threshold, int32_t max_iter, int32_t patch_half, const int32_t *window, float *model,
              int32_t *n_iter, void *stream) {
    CL_GUARD_BEGIN
    if (!ctx || !residual || !psf || !model || !n_iter) return aw_set_error(AW_EINVAL, "NULL argument");
    if (npol != 1 && npol != 4) return aw_set_error(AW_EINVAL, "npol %d", npol);
    if (N < 4 || (int64_t)N * N > 0xFFFFFFFFll) return aw_set_error(AW_EINVAL, "N=%d", N);
    if (!(gain > 0.f && gain <= 1.f)) return aw_set_error(AW_EINVAL, "gain %g outside (0, 1]", (double)gain);
    if (max_iter < 0) return aw_set_error(AW_EINVAL, "max_iter %d", max_iter);
    if (patch_half < 0 || patch_half >= N / 2) return aw_set_error(AW_EINVAL, "patch_half %d", patch_half);
    int rc = check_window(window, N);
    if (rc) return rc;
    rc = use_device(ctx->device);
    if (rc) return rc;
    return hogbom_impl(ctx, residual, psf, npol, N, gain, threshold, max_iter, patch_half, window, model, n_iter,
                       S_(stream));
    CL_GUARD_END
}

int aw_grid_batched(aw_ctx *ctx, aw_plan *p, const aw_kernel_set *k, const void *vis, const float *weight,
                    void *grid, aw_stats *stats, void *stream);

int aw_clean(aw_ctx *ctx, aw_plan *p, const aw_kernel_set *kg, const aw_kernel_set *kd, const void *vis,
             const float *weight, const aw_clean_cfg *cfg, float *model, float *residual, float *psf,
             aw_clean_report *report, void *stream) {
    CL_GUARD_BEGIN
    if (!ctx || !cfg || !model || !residual || !psf || !report) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = check_plan_kset(p, kg);
    if (rc) return rc;
    rc = check_plan_kset(p, kd);
    if (rc) return rc;
    if (kg->spec.role != AW_ROLE_GRID) return aw_set_error(AW_EINVAL, "kgrid is not a GRID kernel set");
    if (kd->spec.role == AW_ROLE_GRID) return aw_set_error(AW_EINVAL, "kdegrid is a GRID kernel set");
    if (!vis && p->nvis) return aw_set_error(AW_EINVAL, "vis is NULL");
    const int N = p->N, npol = p->npol;
    if (cfg->n_major < 1 || cfg->max_minor < 0 || !(cfg->gain > 0.f && cfg->gain <= 1.f) ||
        !(cfg->cycle_factor >= 0.f) || cfg->patch_half < 0 || cfg->patch_half >= N / 2)
        return aw_set_error(AW_EINVAL, "clean configuration out of range");
    int32_t win[4] = {cfg->window[0], cfg->window[1], cfg->window[2], cfg->window[3]};
    if (!win[0] && !win[1] && !win[2] && !win[3]) {
        win[0] = win[1] = N / 4;
        win[2] = win[3] = 3 * N / 4;
    }
    rc = check_window(win, N);
    if (rc) return rc;
    rc = use_device(ctx->device);
    if (rc) return rc;
    cudaStream_t s = S_(stream);
    const int64_t plane = (int64_t)N * N;
    const size_t vbytes = sizeof(float2) * (size_t)npol * (size_t)std::max<int64_t>(p->nvis, 1);
    DevMem rv, gr;
    AW_CUDA_TRY(aw_dev_malloc(&rv.p, vbytes));
    AW_CUDA_TRY(aw_dev_malloc(&gr.p, sizeof(float2) * (size_t)npol * plane));
    float2 *res_vis = reinterpret_cast<float2 *>(rv.p);
    aw_clean_report rep{};
    aw_stats st{};
    // point-spread function: unit Stokes I visibilities, same weights and kernels
    unit_vis_kernel<<<nblk(p->nvis * npol, 256), 256, 0, s>>>(res_vis, p->nvis, npol);
    AW_CHECK_LAUNCH();
    AW_CUDA_TRY(cudaMemsetAsync(gr.p, 0, sizeof(float2) * (size_t)npol * plane, s));
    rc = aw_grid_batched(ctx, p, kg, res_vis, weight, gr.p, &st, stream);
    if (rc) return rc;
    if (!(st.weight_sum > 0)) return aw_set_error(AW_EINVAL, "no visibility was gridded (weight sum %g)", st.weight_sum);
    rep.weight_sum = st.weight_sum;
    rc = aw_fft_to_image_impl(ctx, N, npol, kg->spec.W, gr.p, st.weight_sum, residual, s);
    if (rc) return rc;
    psf_norm_kernel<<<nblk(plane, 256), 256, 0, s>>>(residual, N, psf);
    AW_CHECK_LAUNCH();
    rc = sidelobe_impl(ctx, psf, N, &rep.sidelobe, s);
    if (rc) return rc;
    // major cycles
    AW_CUDA_TRY(cudaMemsetAsync(model, 0, sizeof(float) * (size_t)npol * plane, s));
    AW_CUDA_TRY(cudaMemcpyAsync(res_vis, vis, vbytes, cudaMemcpyDeviceToDevice, s));
    bool stopped = false;
    for (int k = 0; k < cfg->n_major; ++k) {
        AW_CUDA_TRY(cudaMemsetAsync(gr.p, 0, sizeof(float2) * (size_t)npol * plane, s));
        rc = aw_grid_batched(ctx, p, kg, res_vis, weight, gr.p, &st, stream);
        if (rc) return rc;
        rc = aw_fft_to_image_impl(ctx, N, npol, kg->spec.W, gr.p, st.weight_sum, residual, s);
        if (rc) return rc;
        float peak = 0.f;
        rc = window_peak_impl(ctx, residual, N, win, &peak, s);
        if (rc) return rc;
        if (k == 0) rep.peak_first = peak;
        rep.peak_last = peak;
        if (peak < cfg->threshold) { stopped = true; break; }
        const float thr = std::max(cfg->threshold, (cfg->cycle_factor * rep.sidelobe) * peak);
        int32_t n = 0;
        rc = hogbom_impl(ctx, residual, psf, npol, N, cfg->gain, thr, cfg->max_minor, cfg->patch_half, win, model,
                         &n, s);
        if (rc) return rc;
        rep.n_minor += n;
        rep.n_major += 1;
        rc = aw_image_to_grid_impl(ctx, N, npol, kd->spec.W, model, gr.p, s);
        if (rc) return rc;
        rc = aw_launch_degrid(p, kd, gr.p, res_vis, s, vis);
        if (rc) return rc;
    }
    if (!stopped) {
        // the residual image of the last prediction
        AW_CUDA_TRY(cudaMemsetAsync(gr.p, 0, sizeof(float2) * (size_t)npol * plane, s));
        rc = aw_grid_batched(ctx, p, kg, res_vis, weight, gr.p, &st, stream);
        if (rc) return rc;
        rc = aw_fft_to_image_impl(ctx, N, npol, kg->spec.W, gr.p, st.weight_sum, residual, s);
        if (rc) return rc;
        rc = window_peak_impl(ctx, residual, N, win, &rep.peak_last, s);
        if (rc) return rc;
    }
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    *report = rep;
    return AW_OK;
    CL_GUARD_END
}

}  // extern "C"
