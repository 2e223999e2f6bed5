// C ABI entry points of libaw (declared in include/aw.h): argument checks,
// handle management, and dispatch to the kernels of the other units.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "aw_internal.h"

int aw_kernel_set_geometry(const aw_kernel_spec *spec, aw_kernel_set *ks);
int aw_kernel_set_alloc(aw_kernel_set *ks);
int aw_synthesise(aw_ctx *ctx, aw_kernel_set *ks, cudaStream_t s);
int aw_plan_build(aw_ctx *ctx, const aw_vis_desc *vis, const aw_kernel_set *ks, const aw_tune *tune,
                  aw_plan *plan, cudaStream_t s);
int aw_plan_coords_impl(const aw_plan *plan, const aw_kernel_set *ks, int32_t *x0, int32_t *y0,
                        int32_t *fx, int32_t *fy, int32_t *bin, uint8_t *flip, uint8_t *valid,
                        cudaStream_t s);
int aw_plan_order_impl(const aw_plan *plan, uint32_t *perm, cudaStream_t s);
int aw_fft_to_image_impl(aw_ctx *ctx, int N, int npol, double W, void *grid, double weight_sum,
                         float *image, cudaStream_t s);
int aw_mosaic_gamma_impl(aw_ctx *ctx, const float *beams, int nfield, int N, float eps, float *gamma,
                         cudaStream_t s);

static thread_local char g_err[1024] = "";

// ---------------------------------------------------------------- device memory hook
static std::atomic<long long> g_alloc_calls{0};   // device allocations attempted
static std::atomic<long long> g_alloc_live{0};    // buffers allocated and not freed
static std::atomic<long long> g_alloc_fail_at{-1};  // g_alloc_calls value that fails, or -1

cudaError_t aw_dev_malloc_raw(void **p, size_t bytes) {
    const long long k = g_alloc_calls.fetch_add(1);
    if (k == g_alloc_fail_at.load()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;   // injected: nothing was allocated
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_alloc_live.fetch_add(1);
    return e;
}

void aw_dev_free(void *p) {
    if (!p) return;
    cudaFree(p);
    g_alloc_live.fetch_sub(1);
}

int aw_set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define AW_GUARD_BEGIN \
    AW_TRACE();         \
    try {
#define AW_GUARD_END                                                   \
    }                                                                  \
    catch (const std::bad_alloc &) {                                   \
        return aw_set_error(AW_ENOMEM, "host allocation failed");      \
    }                                                                  \
    catch (...) {                                                      \
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");    \
    }

static inline cudaStream_t S_(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static int use_device(int dev) {
    int cur = -1;
    AW_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != dev) AW_CUDA_TRY(cudaSetDevice(dev));
    return AW_OK;
}

int aw_ctx_fft_plan(aw_ctx *ctx, int rank_tag, int n, int batch, cufftType type, cufftHandle *out) {
    auto key = std::make_tuple(rank_tag, n, batch, (int)type);
    auto it = ctx->fft_plans.find(key);
    if (it != ctx->fft_plans.end()) { *out = it->second; return AW_OK; }
    cufftHandle h;
    int dims[2] = {n, n};
    AW_CUFFT_TRY(cufftPlanMany(&h, 2, dims, nullptr, 1, n * n, nullptr, 1, n * n, type, batch));
    ctx->fft_plans[key] = h;
    *out = h;
    return AW_OK;
}

extern "C" {

const char *aw_last_error(void) { return g_err; }

int aw_create(aw_ctx **ctx, int device) {
    AW_GUARD_BEGIN
    if (!ctx) return aw_set_error(AW_EINVAL, "ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    AW_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return aw_set_error(AW_EINVAL, "device %d of %d", device, ndev);
    AW_CUDA_TRY(cudaSetDevice(device));
    aw_ctx *c = new aw_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = aw_dev_malloc(&c->d_scratch, 256);
    if (e != cudaSuccess) {
        delete c;
        return aw_set_error(AW_ENOMEM, "context scratch: %s", cudaGetErrorString(e));
    }
    *ctx = c;
    return AW_OK;
    AW_GUARD_END
}

int aw_destroy(aw_ctx *ctx) {
    AW_GUARD_BEGIN
    if (!ctx) return AW_OK;
    use_device(ctx->device);
    for (auto &kv : ctx->fft_plans) cufftDestroy(kv.second);
    for (auto &kv : ctx->gridcorr) aw_dev_free(kv.second);
    if (ctx->d_scratch) aw_dev_free(ctx->d_scratch);
    delete ctx;
    return AW_OK;
    AW_GUARD_END
}

static void free_kset(aw_kernel_set *k) {
    if (!k) return;
    if (k->d_table) aw_dev_free(k->d_table);
    if (k->d_bin_support) aw_dev_free(k->d_bin_support);
    if (k->d_bin_offset) aw_dev_free(k->d_bin_offset);
    delete k;
}

int aw_make_kernels(aw_ctx *ctx, const aw_kernel_spec *spec, aw_kernel_set **out, void *stream) {
    AW_GUARD_BEGIN
    if (!ctx || !out) return aw_set_error(AW_EINVAL, "ctx/out is NULL");
    *out = nullptr;
    int rc = use_device(ctx->device);
    if (rc) return rc;
    aw_kernel_set *k = new aw_kernel_set();
    k->device = ctx->device;
    rc = aw_kernel_set_geometry(spec, k);
    if (rc == AW_OK) rc = aw_kernel_set_alloc(k);
    if (rc == AW_OK) rc = aw_synthesise(ctx, k, S_(stream));
    if (rc != AW_OK) { free_kset(k); return rc; }
    *out = k;
    return AW_OK;
    AW_GUARD_END
}

int aw_kernel_set_import(aw_ctx *ctx, const aw_kernel_spec *spec, const void *tables, aw_kernel_set **out,
                         void *stream) {
    AW_GUARD_BEGIN
    if (!ctx || !out || !tables) return aw_set_error(AW_EINVAL, "ctx/out/tables is NULL");
    *out = nullptr;
    int rc = use_device(ctx->device);
    if (rc) return rc;
    aw_kernel_set *k = new aw_kernel_set();
    k->device = ctx->device;
    rc = aw_kernel_set_geometry(spec, k);
    if (rc == AW_OK) rc = aw_kernel_set_alloc(k);
    if (rc == AW_OK && k->spec.storage == AW_STORAGE_FP16) {
        float mx = 0.f;
        rc = aw_table_absmax(reinterpret_cast<const float2 *>(tables), k->total_elems, &mx, S_(stream));
        if (rc == AW_OK && mx > 0.f) k->scale = (float)std::ldexp(1.0, (int)std::floor(-std::log2((double)mx)));
    }
    for (int b = 0; rc == AW_OK && b < k->nbins; ++b) {
        const int S = k->bin_support[b];
        const char *src = static_cast<const char *>(tables) + k->bin_offset[b] * sizeof(float2);
        char *dst = static_cast<char *>(k->d_table) + k->bin_offset[b] * k->elem_bytes;
        rc = aw_convert_table_scaled(reinterpret_cast<const float2 *>(src), dst, (int64_t)k->spec.OS * k->spec.OS,
                                     S * S, k->P, k->ce, k->spec.storage, k->scale, S_(stream));
    }
    if (rc == AW_OK) {
        cudaError_t e = cudaStreamSynchronize(S_(stream));
        if (e != cudaSuccess) rc = aw_set_error(AW_ECUDA, "import: %s", cudaGetErrorString(e));
    }
    if (rc != AW_OK) { free_kset(k); return rc; }
    *out = k;
    return AW_OK;
    AW_GUARD_END
}

int aw_kernel_set_export(const aw_kernel_set *k, int32_t bin, void *dst, void *stream) {
    AW_GUARD_BEGIN
    if (!k || !dst) return aw_set_error(AW_EINVAL, "kset/dst is NULL");
    if (bin < 0 || bin >= k->nbins) return aw_set_error(AW_EINVAL, "bin %d of %d", bin, k->nbins);
    int rc = use_device(k->device);
    if (rc) return rc;
    const int S = k->bin_support[bin];
    const int64_t n = (int64_t)k->spec.OS * k->spec.OS * S * S * k->P;
    const char *src = static_cast<const char *>(k->d_table) + k->bin_offset[bin] * k->elem_bytes;
    (void)n;
    return aw_export_table(src, reinterpret_cast<float2 *>(dst), (int64_t)k->spec.OS * k->spec.OS, S * S, k->P,
                           k->ce, k->spec.storage, 1.0f / k->scale, S_(stream));
    AW_GUARD_END
}

int aw_kernel_set_info(const aw_kernel_set *k, aw_kernel_info *info) {
    if (!k || !info) return aw_set_error(AW_EINVAL, "kset/info is NULL");
    info->bytes = k->total_elems * k->elem_bytes;
    info->nbins = k->nbins;
    info->max_support = k->max_support;
    info->npol = k->spec.npol;
    info->role = k->spec.role;
    info->storage = k->spec.storage;
    info->N = k->spec.N;
    info->OS = k->spec.OS;
    info->n_rejected = k->n_rejected;
    return AW_OK;
}

int aw_kernel_set_destroy(aw_kernel_set *k) {
    AW_GUARD_BEGIN
    if (!k) return AW_OK;
    use_device(k->device);
    free_kset(k);
    return AW_OK;
    AW_GUARD_END
}

static void free_plan(aw_plan *p) {
    if (!p) return;
    p->drop_graphs();
    if (p->d_rec) aw_dev_free(p->d_rec);
    if (p->d_items) aw_dev_free(p->d_items);
    if (p->d_rec_dg) aw_dev_free(p->d_rec_dg);
    if (p->d_items_dg) aw_dev_free(p->d_items_dg);
    if (p->d_plane_support) aw_dev_free(p->d_plane_support);
    if (p->d_wsum) aw_dev_free(p->d_wsum);
    if (p->d_nonfinite) aw_dev_free(p->d_nonfinite);
    if (p->d_counter) aw_dev_free(p->d_counter);
    if (p->d_items_ht) aw_dev_free(p->d_items_ht);
    if (p->d_items_ho) aw_dev_free(p->d_items_ho);
    if (p->d_rec_rg) aw_dev_free(p->d_rec_rg);
    for (auto &c : p->rclasses)
        if (c.d_items) aw_dev_free(c.d_items);
    if (p->d_rcounter) aw_dev_free(p->d_rcounter);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->aux) cudaStreamDestroy(p->aux);
    delete p;
}

int aw_plan_create(aw_ctx *ctx, const aw_vis_desc *vis, const aw_kernel_set *kset, const aw_tune *tune,
                   aw_plan **out, void *stream) {
    AW_GUARD_BEGIN
    if (!ctx || !kset || !out) return aw_set_error(AW_EINVAL, "ctx/kset/out is NULL");
    *out = nullptr;
    int rc = use_device(ctx->device);
    if (rc) return rc;
    aw_plan *p = new aw_plan();
    p->device = ctx->device;
    aw_tune cached{};
    if (!tune && ctx->has_tune) {
        // a cached split names planes of the set it was tuned on: a hybrid split
        // without planes of this set on both sides of it, or a region split past
        // this set's planes, takes the offset schedule instead (a set of another
        // plane layout was not tuned; the offset kernel suits any layout)
        cached = ctx->tune_cache;
        if (cached.grid_mode == AW_GRID_HYBRID && (cached.split_planes < 1 || cached.split_planes >= kset->spec.nw))
            cached.grid_mode = AW_GRID_OFFSETS;
        if (cached.grid_mode == AW_GRID_REGION && cached.split_planes > kset->spec.nw)
            cached.grid_mode = AW_GRID_OFFSETS;
        tune = &cached;
    }
    rc = aw_plan_build(ctx, vis, kset, tune, p, S_(stream));
    if (rc != AW_OK) { free_plan(p); return rc; }
    *out = p;
    return AW_OK;
    AW_GUARD_END
}

int aw_plan_query(const aw_plan *p, aw_plan_info *info) {
    if (!p || !info) return aw_set_error(AW_EINVAL, "plan/info is NULL");
    info->nvis = p->nvis;
    info->nvalid = p->nvalid;
    info->n_outside = p->n_outside;
    info->n_flagged = p->n_flagged;
    info->nitems = p->nitems;
    info->tile = p->tune.tile;
    info->chunk = p->tune.chunk;
    info->mean_taps = p->mean_taps;
    info->nitems_degrid = p->nitems_dg;
    int nl = 0;
    for (const auto &c : p->rclasses) nl += c.n > 0;
    info->region_lists = nl;
    switch (p->tune.grid_mode) {
        case AW_GRID_HYBRID: info->grid_kernels = (p->nitems_ht > 0) + (p->nitems_ho > 0); break;
        case AW_GRID_REGION: info->grid_kernels = nl + (p->nitems_ho > 0); break;
        default: info->grid_kernels = p->nitems > 0 ? 1 : 0;
    }
    return AW_OK;
}

int aw_plan_destroy(aw_plan *p) {
    AW_GUARD_BEGIN
    if (!p) return AW_OK;
    use_device(p->device);
    free_plan(p);
    return AW_OK;
    AW_GUARD_END
}

int aw_plan_coords(const aw_plan *p, int32_t *x0, int32_t *y0, int32_t *fx, int32_t *fy, int32_t *bin,
                   uint8_t *flip, uint8_t *valid, void *stream) {
    AW_GUARD_BEGIN
    if (!p) return aw_set_error(AW_EINVAL, "plan is NULL");
    int rc = use_device(p->device);
    if (rc) return rc;
    return aw_plan_coords_impl(p, nullptr, x0, y0, fx, fy, bin, flip, valid, S_(stream));
    AW_GUARD_END
}

int aw_plan_order(const aw_plan *p, uint32_t *perm, void *stream) {
    AW_GUARD_BEGIN
    if (!p || !perm) return aw_set_error(AW_EINVAL, "plan/perm is NULL");
    int rc = use_device(p->device);
    if (rc) return rc;
    return aw_plan_order_impl(p, perm, S_(stream));
    AW_GUARD_END
}

static int check_pair(const aw_plan *p, const aw_kernel_set *k) {
    if (!p || !k) return aw_set_error(AW_EINVAL, "plan/kset is NULL");
    if (p->N != k->spec.N || p->OS != k->spec.OS || p->npol != k->spec.npol || p->nbins != k->nbins || p->ntype != k->ntype ||
        p->bin_support != k->bin_support)
        return aw_set_error(AW_EINVAL, "kernel set geometry does not match the plan");
    return AW_OK;
}

static int fill_stats(const aw_plan *p, aw_stats *stats, cudaStream_t s) {
    double ws = 0;
    unsigned long long nb = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&ws, p->d_wsum, sizeof(double), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaMemcpyAsync(&nb, p->d_nonfinite, sizeof(nb), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    stats->n_nonfinite = (int64_t)nb;
    stats->n_gridded = p->nvalid - (int64_t)nb;
    stats->n_outside = p->n_outside;
    stats->n_flagged = p->n_flagged;
    stats->weight_sum = ws;
    return AW_OK;
}

// The plan's gridding schedule on stream s.  AW_GRID_HYBRID forks: the TILES
// part (persistent, its d_counter zeroed by the caller) runs on s, the OFFSETS
// part on the plan's second stream, sized to fit beside the TILES CTAs, and s
// then waits for both; inside a stream capture the fork and join become edges
// of the graph.
static int launch_planned(aw_ctx *ctx, const aw_plan *p, const aw_kernel_set *k, const void *vis,
                          const float *weight, void *grid, bool persistent, cudaStream_t s) {
    auto ctas_for = [&](int64_t n) {
        const int64_t c = std::min<int64_t>((int64_t)ctx->sm_count * p->tune.ctas_per_sm, n);
        return (int)std::max<int64_t>(c, 1);
    };
    if (p->tune.grid_mode == AW_GRID_REGION) {
        // the region lists on the caller's stream; the bins that take no region
        // (wide supports, or planes from split_planes on) with the OFFSETS
        // kernel on the second stream at the same time, one CTA per SM (it
        // fits beside two region CTAs: registers, shared memory, threads)
        if (p->nitems_ho == 0) return aw_launch_grid_region(p, k, vis, weight, grid, s);
        if (p->nreg == 0) {   // no bin takes a region: OFFSETS alone, every SM
            aw_grid_launch Lo{p, k, vis, weight, grid, false, 0, s, AW_GRID_OFFSETS, p->d_items_ho, p->nitems_ho};
            return aw_launch_grid(Lo);
        }
        if (!p->aux) return aw_set_error(AW_EINVAL, "region plan without its second stream");
        AW_CUDA_TRY(cudaEventRecord(p->ev_fork, s));
        AW_CUDA_TRY(cudaStreamWaitEvent(p->aux, p->ev_fork, 0));
        aw_grid_launch Lo{p, k, vis, weight, grid, false, ctx->sm_count, p->aux, AW_GRID_OFFSETS, p->d_items_ho,
                          p->nitems_ho};
        int rc = aw_launch_grid(Lo);
        if (rc == AW_OK) rc = aw_launch_grid_region(p, k, vis, weight, grid, s);
        AW_CUDA_TRY(cudaEventRecord(p->ev_join, p->aux));
        AW_CUDA_TRY(cudaStreamWaitEvent(s, p->ev_join, 0));
        return rc;
    }
    if (p->tune.grid_mode != AW_GRID_HYBRID) {
        aw_grid_launch L{p, k, vis, weight, grid, persistent, ctas_for(p->nitems), s};
        return aw_launch_grid(L);
    }
    if (p->nitems == 0) return AW_OK;
    if (!p->aux) return aw_set_error(AW_EINVAL, "hybrid plan without its second stream");
    AW_CUDA_TRY(cudaEventRecord(p->ev_fork, s));
    AW_CUDA_TRY(cudaStreamWaitEvent(p->aux, p->ev_fork, 0));
    aw_grid_launch Lt{p, k, vis, weight, grid, true, ctas_for(p->nitems_ht), s,
                      AW_GRID_TILES, p->d_items_ht, p->nitems_ht};
    int rc = aw_launch_grid(Lt);
    if (rc == AW_OK) {
        aw_grid_launch Lo{p, k, vis, weight, grid, false, 0, p->aux, AW_GRID_OFFSETS, p->d_items_ho, p->nitems_ho};
        rc = aw_launch_grid(Lo);
    }
    // joined even after a failed launch, so that a capture is not left forked
    AW_CUDA_TRY(cudaEventRecord(p->ev_join, p->aux));
    AW_CUDA_TRY(cudaStreamWaitEvent(s, p->ev_join, 0));
    return rc;
}

int aw_grid(aw_ctx *ctx, const aw_plan *p, const aw_kernel_set *k, const void *vis, const float *weight,
            void *grid, aw_stats *stats, void *stream) {
    AW_GUARD_BEGIN
    if (!ctx) return aw_set_error(AW_EINVAL, "ctx is NULL");
    int rc = check_pair(p, k);
    if (rc) return rc;
    if ((!vis && p->nvis) || !grid) return aw_set_error(AW_EINVAL, "vis/grid is NULL");
    rc = use_device(ctx->device);
    if (rc) return rc;
    cudaStream_t s = S_(stream);
    AW_CUDA_TRY(cudaMemsetAsync(p->d_wsum, 0, sizeof(double), s));
    AW_CUDA_TRY(cudaMemsetAsync(p->d_nonfinite, 0, sizeof(unsigned long long), s));
    if (p->tune.grid_mode == AW_GRID_HYBRID) AW_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int), s));
    rc = launch_planned(ctx, p, k, vis, weight, grid, false, s);
    if (rc) return rc;
    if (stats) return fill_stats(p, stats, s);
    return AW_OK;
    AW_GUARD_END
}

int aw_degrid(aw_ctx *ctx, const aw_plan *p, const aw_kernel_set *k, const void *grid, void *vis_out,
              void *stream) {
    AW_GUARD_BEGIN
    if (!ctx) return aw_set_error(AW_EINVAL, "ctx is NULL");
    int rc = check_pair(p, k);
    if (rc) return rc;
    if (!grid || (!vis_out && p->nvis)) return aw_set_error(AW_EINVAL, "grid/vis_out is NULL");
    rc = use_device(ctx->device);
    if (rc) return rc;
    return aw_launch_degrid(p, k, grid, vis_out, S_(stream));
    AW_GUARD_END
}

int aw_grid_batched(aw_ctx *ctx, aw_plan *p, const aw_kernel_set *k, const void *vis, const float *weight,
                    void *grid, aw_stats *stats, void *stream) {
    AW_GUARD_BEGIN
    if (!ctx) return aw_set_error(AW_EINVAL, "ctx is NULL");
    int rc = check_pair(p, k);
    if (rc) return rc;
    if ((!vis && p->nvis) || !grid) return aw_set_error(AW_EINVAL, "vis/grid is NULL");
    rc = use_device(ctx->device);
    if (rc) return rc;
    cudaStream_t s = S_(stream);
    if (p->nitems == 0) {
        AW_CUDA_TRY(cudaMemsetAsync(p->d_wsum, 0, sizeof(double), s));
        AW_CUDA_TRY(cudaMemsetAsync(p->d_nonfinite, 0, sizeof(unsigned long long), s));
        if (stats) return fill_stats(p, stats, s);
        return AW_OK;
    }
    aw_plan::GraphSlot *slot = nullptr;
    for (auto &g : p->gslots)
        if (g.exec && g.vis == vis && g.weight == weight && g.grid == grid && g.kset == k && g.stream == s) slot = &g;
    if (!slot) {
        slot = p->gslots[0].used <= p->gslots[1].used ? &p->gslots[0] : &p->gslots[1];
        if (slot->exec) { cudaGraphExecDestroy(slot->exec); *slot = aw_plan::GraphSlot{}; }
        cudaStream_t cap;
        AW_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaMemsetAsync(p->d_wsum, 0, sizeof(double), cap);
            cudaMemsetAsync(p->d_nonfinite, 0, sizeof(unsigned long long), cap);
            cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int), cap);
            rc = launch_planned(ctx, p, k, vis, weight, grid, true, cap);
            e = cudaStreamEndCapture(cap, &g);
        }
        if (e == cudaSuccess && rc == AW_OK) e = cudaGraphInstantiate(&slot->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (rc) return rc;
        if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        slot->vis = vis;
        slot->weight = weight;
        slot->grid = grid;
        slot->kset = k;
        slot->stream = s;
    }
    slot->used = ++p->gclock;
    AW_CUDA_TRY(cudaGraphLaunch(slot->exec, s));
    if (stats) return fill_stats(p, stats, s);
    return AW_OK;
    AW_GUARD_END
}

int aw_autotune(aw_ctx *ctx, const aw_vis_desc *vis, const aw_kernel_set *k, aw_tune *out, void *stream) {
    AW_GUARD_BEGIN
    if (!ctx || !vis || !k || !out) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = use_device(ctx->device);
    if (rc) return rc;
    cudaStream_t s = S_(stream);
    const size_t gbytes = sizeof(float2) * (size_t)k->spec.npol * k->spec.N * k->spec.N;
    void *grid = nullptr, *v = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&grid, gbytes));
    cudaError_t e = aw_dev_malloc(&v, sizeof(float2) * (size_t)k->spec.npol * std::max<int64_t>(vis->nvis, 1));
    if (e != cudaSuccess) { aw_dev_free(grid); return aw_set_error(AW_ENOMEM, "autotune vis buffer"); }
    cudaMemsetAsync(v, 0, sizeof(float2) * (size_t)k->spec.npol * std::max<int64_t>(vis->nvis, 1), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tiles[] = {16, 32, 64};
    const int chunks[] = {128, 256, 512};
    const int ctas[] = {2, 4, 5};
    float best = 1e30f;
    aw_tune bt{32, 256, 2, 0, AW_GRID_TILES};
    // one timing of aw_grid_batched on plan p: best of reps 2..3
    auto time_plan = [&](aw_plan *p, float *ms_out) -> int {
        p->drop_graphs();
        float ms_best = 1e30f;
        int r = AW_OK;
        for (int rep = 0; rep < 3 && r == AW_OK; ++rep) {
            cudaMemsetAsync(grid, 0, gbytes, s);
            cudaEventRecord(e0, s);
            r = aw_grid_batched(ctx, p, k, v, nullptr, grid, nullptr, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < ms_best) ms_best = ms;
        }
        *ms_out = ms_best;
        return r;
    };
    for (int t : tiles) {
        for (int c : chunks) {
            aw_tune tu{t, c, 1, 0, AW_GRID_TILES};
            aw_plan *p = new aw_plan();
            p->device = ctx->device;
            rc = aw_plan_build(ctx, vis, k, &tu, p, s);
            if (rc) { free_plan(p); break; }
            for (int cp : ctas) {
                p->tune.ctas_per_sm = cp;
                float ms_best = 1e30f;
                rc = time_plan(p, &ms_best);
                if (rc) break;
                if (ms_best < best) { best = ms_best; bt = aw_tune{t, c, cp, 0, AW_GRID_TILES}; }
            }
            free_plan(p);
            if (rc) break;
        }
        if (rc) break;
    }
    // the offset-grouped schedule, over two super-tile sizes
    const int dg_tiles[] = {256, 1024};
    for (int dt : dg_tiles) {
        if (rc) break;
        aw_tune tu{bt.tile, bt.chunk, bt.ctas_per_sm, dt, AW_GRID_OFFSETS};
        aw_plan *p = new aw_plan();
        p->device = ctx->device;
        rc = aw_plan_build(ctx, vis, k, &tu, p, s);
        if (rc) { free_plan(p); break; }
        float ms_best = 1e30f;
        rc = time_plan(p, &ms_best);
        free_plan(p);
        if (rc) break;
        if (ms_best < best) { best = ms_best; bt = tu; }
    }
    // the region schedule: the w planes up to the last one whose support is at
    // most 32, 40 or 48 cells on the region kernel (bins whose support has no
    // region form stay on OFFSETS), the rest on OFFSETS at the same time (its
    // super-tile the larger one)
    if (!rc) {
        int last_split = -1;
        for (int lim : {32, 40, 48}) {
            int q = 0;
            while (q < k->spec.nw && k->supports[(size_t)q] <= lim) ++q;
            if (q == 0 || q == last_split) continue;
            last_split = q;
            aw_tune tu{bt.tile, bt.chunk, 2, 1024, AW_GRID_REGION, q};
            aw_plan *p = new aw_plan();
            p->device = ctx->device;
            int r2 = aw_plan_build(ctx, vis, k, &tu, p, s);
            float ms_best = 1e30f;
            if (!r2) r2 = time_plan(p, &ms_best);
            free_plan(p);
            if (!r2 && ms_best < best) { best = ms_best; bt = tu; }
            if (r2) cudaGetLastError();   // a candidate that cannot be built is skipped
        }
    }
    // the hybrid schedule: the first planes holding about a quarter to a half
    // of the visibility-taps on TILES, the rest on OFFSETS, at 2 or 3 TILES CTAs
    // per SM.  A hybrid candidate that cannot be built or run (its second stream
    // or events, its item lists) is skipped: the TILES / OFFSETS schedule
    // already measured stays the answer.
    std::vector<double> cum;
    int hrc = rc;
    if (!hrc) {
        aw_tune tu{bt.tile, bt.chunk, 2, bt.dg_tile ? bt.dg_tile : 1024, AW_GRID_TILES};
        aw_plan *p = new aw_plan();
        p->device = ctx->device;
        hrc = aw_plan_build(ctx, vis, k, &tu, p, s);
        if (!hrc) hrc = aw_plan_plane_taps(p, cum, s);
        free_plan(p);
    }
    int last_q = -1;
    const double targets[] = {0.25, 0.35, 0.45};
    for (double target : targets) {
        if (hrc || cum.empty()) break;
        int q = 1;
        while (q < (int)cum.size() - 1 && cum[q] < target) ++q;   // cum[q]: share of planes < q
        if (q <= last_q || q >= (int)cum.size() - 1) continue;
        last_q = q;
        aw_tune tu{bt.tile, bt.chunk, 2, bt.dg_tile ? bt.dg_tile : 1024, AW_GRID_HYBRID, q};
        aw_plan *p = new aw_plan();
        p->device = ctx->device;
        hrc = aw_plan_build(ctx, vis, k, &tu, p, s);
        if (hrc) { free_plan(p); break; }
        for (int cp : {2, 3}) {
            p->tune.ctas_per_sm = cp;
            float ms_best = 1e30f;
            hrc = time_plan(p, &ms_best);
            if (hrc) break;
            if (ms_best < best) { best = ms_best; bt = p->tune; }
        }
        free_plan(p);
    }
    if (hrc && !rc) cudaGetLastError();   // clear a non-sticky error of the skipped candidate
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    aw_dev_free(grid);
    aw_dev_free(v);
    if (rc) return rc;
    *out = bt;
    ctx->tune_cache = bt;
    ctx->has_tune = true;
    return AW_OK;
    AW_GUARD_END
}

int aw_fft_to_image(aw_ctx *ctx, const aw_kernel_set *k, void *grid, double weight_sum, float *image,
                    void *stream) {
    AW_GUARD_BEGIN
    if (!ctx || !k || !grid || !image) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = use_device(ctx->device);
    if (rc) return rc;
    return aw_fft_to_image_impl(ctx, k->spec.N, k->spec.npol, k->spec.W, grid, weight_sum, image, S_(stream));
    AW_GUARD_END
}

int mosaic_gamma(aw_ctx *ctx, const float *beams, int32_t nfield, int32_t N, float eps, float *gamma,
                 void *stream) {
    AW_GUARD_BEGIN
    if (!ctx || !beams || !gamma) return aw_set_error(AW_EINVAL, "NULL argument");
    if (nfield < 1 || N < 1) return aw_set_error(AW_EINVAL, "nfield=%d N=%d", nfield, N);
    int rc = use_device(ctx->device);
    if (rc) return rc;
    return aw_mosaic_gamma_impl(ctx, beams, nfield, N, eps, gamma, S_(stream));
    AW_GUARD_END
}

}  // extern "C"

// ---------------------------------------------------------------- failure injection and self-tests
int aw_barrier_selftest(aw_ctx *ctx, cudaStream_t s);
int aw_mbar_selftest(cudaStream_t st);

extern "C" int aw_debug_fail_alloc(int64_t n) {
    if (n < -1) return aw_set_error(AW_EINVAL, "n = %lld", (long long)n);
    g_alloc_fail_at.store(n < 0 ? -1 : g_alloc_calls.load() + n);
    return AW_OK;
}

extern "C" int aw_debug_alloc_stats(int64_t *live, int64_t *calls) {
    if (!live || !calls) return aw_set_error(AW_EINVAL, "NULL argument");
    *live = g_alloc_live.load();
    *calls = g_alloc_calls.load();
    return AW_OK;
}

extern "C" int aw_debug_wait_timeout(aw_ctx *ctx, int32_t which, void *stream) {
    AW_GUARD_BEGIN
    if (!ctx) return aw_set_error(AW_EINVAL, "ctx is NULL");
    int rc = use_device(ctx->device);
    if (rc) return rc;
    if (which == 0) return aw_barrier_selftest(ctx, S_(stream));
    if (which == 1) return aw_mbar_selftest(S_(stream));
    return aw_set_error(AW_EINVAL, "which = %d", which);
    AW_GUARD_END
}
