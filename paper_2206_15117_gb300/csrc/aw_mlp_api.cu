// C ABI entry points of the learned kernel surrogate (include/aw.h).
#include <cstring>
#include <new>

#include "aw_internal.h"
#include "aw_mlp.h"

int aw_kernel_set_geometry(const aw_kernel_spec *spec, aw_kernel_set *ks);
int aw_kernel_set_alloc(aw_kernel_set *ks);

static inline cudaStream_t S_(void *s) { return reinterpret_cast<cudaStream_t>(s); }

#define SUR_GUARD_BEGIN \
    AW_TRACE();         \
    try {
#define SUR_GUARD_END                                                  \
    }                                                                  \
    catch (const std::bad_alloc &) {                                   \
        return aw_set_error(AW_ENOMEM, "host allocation failed");      \
    }                                                                  \
    catch (...) {                                                      \
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");    \
    }

static int set_dev(int d) {
    AW_CUDA_TRY(cudaSetDevice(d));
    return AW_OK;
}

extern "C" {

int aw_surrogate_create(aw_ctx *ctx, const aw_surrogate_cfg *cfg, aw_surrogate **out) {
    SUR_GUARD_BEGIN
    if (!ctx || !cfg || !out) return aw_set_error(AW_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->npol != 1 && cfg->npol != 4) return aw_set_error(AW_EINVAL, "npol %d", cfg->npol);
    if (cfg->width < 8 || cfg->width > 512 || cfg->n_hidden < 1 || cfg->n_hidden > 8)
        return aw_set_error(AW_EINVAL, "width %d / n_hidden %d out of range", cfg->width, cfg->n_hidden);
    if (!(cfg->D > 0) || !(cfg->f_h > 0) || !(cfg->chi_h > 0) || !(cfg->out_scale > 0))
        return aw_set_error(AW_EINVAL, "feature scales must be positive");
    if (cfg->norm_nw < 1 || cfg->norm_nw > 256 || !cfg->norm_supports)
        return aw_set_error(AW_EINVAL, "norm_nw %d / norm_supports", cfg->norm_nw);
    for (int i = 0; i < cfg->norm_nw; ++i)
        if (cfg->norm_supports[i] < 1) return aw_set_error(AW_EINVAL, "norm_supports[%d] < 1", i);
    int rc = set_dev(ctx->device);
    if (rc) return rc;
    aw_surrogate *s = new aw_surrogate();
    s->device = ctx->device;
    s->cfg = *cfg;
    rc = aw_sur_init(s);
    if (rc) {
        aw_sur_free(s);
        delete s;
        return rc;
    }
    *out = s;
    return AW_OK;
    SUR_GUARD_END
}

int aw_surrogate_destroy(aw_surrogate *s) {
    SUR_GUARD_BEGIN
    if (!s) return AW_OK;
    set_dev(s->device);
    aw_sur_free(s);
    delete s;
    return AW_OK;
    SUR_GUARD_END
}

int aw_surrogate_nparams(const aw_surrogate *s, int64_t *n) {
    if (!s || !n) return aw_set_error(AW_EINVAL, "NULL argument");
    *n = s->nparam;
    return AW_OK;
}

int aw_surrogate_set_params(aw_surrogate *s, const float *h) {
    SUR_GUARD_BEGIN
    if (!s || !h) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = set_dev(s->device);
    if (rc) return rc;
    AW_CUDA_TRY(cudaMemcpy(s->d_p, h, sizeof(float) * s->nparam, cudaMemcpyHostToDevice));
    AW_CUDA_TRY(cudaMemset(s->d_m, 0, sizeof(float) * s->nparam));
    AW_CUDA_TRY(cudaMemset(s->d_v, 0, sizeof(float) * s->nparam));
    s->t = 0;
    rc = aw_sur_sync_half(s, 0);
    if (rc) return rc;
    AW_CUDA_TRY(cudaDeviceSynchronize());
    return AW_OK;
    SUR_GUARD_END
}

int aw_surrogate_get_params(const aw_surrogate *s, float *h) {
    SUR_GUARD_BEGIN
    if (!s || !h) return aw_set_error(AW_EINVAL, "NULL argument");
    int rc = set_dev(s->device);
    if (rc) return rc;
    AW_CUDA_TRY(cudaDeviceSynchronize());
    AW_CUDA_TRY(cudaMemcpy(h, s->d_p, sizeof(float) * s->nparam, cudaMemcpyDeviceToHost));
    return AW_OK;
    SUR_GUARD_END
}

int aw_surrogate_forward(aw_ctx *ctx, aw_surrogate *s, const float *X, int32_t B, float *Y, void *stream) {
    SUR_GUARD_BEGIN
    if (!ctx || !s || !X || !Y || B < 0) return aw_set_error(AW_EINVAL, "bad argument");
    if (B == 0) return AW_OK;
    int rc = set_dev(s->device);
    if (rc) return rc;
    rc = aw_sur_alloc_work(s, B);
    if (rc) return rc;
    rc = aw_sur_forward(s, X, B, S_(stream));
    if (rc) return rc;
    AW_CUDA_TRY(cudaMemcpyAsync(Y, s->H.back(), sizeof(float) * (size_t)B * s->sizes.back(), cudaMemcpyDeviceToDevice,
                                S_(stream)));
    return AW_OK;
    SUR_GUARD_END
}

int aw_surrogate_set_train_engine(aw_surrogate *s, int32_t engine) {
    if (!s) return aw_set_error(AW_EINVAL, "surrogate is NULL");
    if (engine != AW_TRAIN_FP32 && engine != AW_TRAIN_TCGEN05) return aw_set_error(AW_EINVAL, "engine %d", engine);
    s->train_engine = engine;
    return AW_OK;
}

int aw_surrogate_loss_grad(aw_ctx *ctx, aw_surrogate *s, const float *X, const float *T, int32_t B, double *loss,
                           float *grad, void *stream) {
    SUR_GUARD_BEGIN
    if (!ctx || !s || !X || !T || !loss || !grad || B <= 0) return aw_set_error(AW_EINVAL, "bad argument");
    int rc = set_dev(s->device);
    if (rc) return rc;
    rc = aw_sur_alloc_work(s, B);
    if (rc) return rc;
    cudaStream_t st = S_(stream);
    double *d_loss = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&d_loss, sizeof(double)));
    cudaMemsetAsync(d_loss, 0, sizeof(double), st);
    if (aw_sur_use_tc(s) && B % 128 == 0) {
        rc = aw_sur_tc_refresh(s, st);
        if (rc == AW_OK) rc = aw_sur_tc_step_grad(s, X, T, B, d_loss, st);
        if (rc == AW_OK) rc = aw_sur_tc_check(s, st);
    } else {
        rc = aw_sur_forward(s, X, B, st);
        if (rc == AW_OK) rc = aw_sur_backward(s, X, T, B, d_loss, st);
    }
    if (rc == AW_OK) {
        cudaError_t e = cudaMemcpyAsync(grad, s->d_g, sizeof(float) * s->nparam, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = aw_set_error(AW_ECUDA, "loss_grad: %s", cudaGetErrorString(e));
    }
    aw_dev_free(d_loss);
    return rc;
    SUR_GUARD_END
}

int aw_surrogate_train(aw_ctx *ctx, aw_surrogate *s, const aw_kernel_set *exact, const aw_train_cfg *cfg,
                       aw_train_report *report, void *stream) {
    SUR_GUARD_BEGIN
    if (!ctx || !s || !exact || !cfg) return aw_set_error(AW_EINVAL, "NULL argument");
    if (cfg->steps < 1 || cfg->batch < 64 || cfg->batch > (1 << 20))
        return aw_set_error(AW_EINVAL, "steps %d / batch %d out of range", cfg->steps, cfg->batch);
    if (exact->nclass > 1) return aw_set_error(AW_EUNSUPPORTED, "the surrogate has no baseline-class input");
    int rc = set_dev(s->device);
    if (rc) return rc;
    return aw_sur_train(s, exact, cfg, report, S_(stream));
    SUR_GUARD_END
}

int aw_surrogate_tables(aw_ctx *ctx, aw_surrogate *s, const aw_kernel_set *exact, float reject_rel, int32_t storage,
                        aw_kernel_set **out, float *bin_err, void *stream) {
    SUR_GUARD_BEGIN
    if (!ctx || !s || !exact || !out) return aw_set_error(AW_EINVAL, "NULL argument");
    *out = nullptr;
    if (exact->P * 2 != s->sizes.back()) return aw_set_error(AW_EINVAL, "surrogate / kernel set npol differ");
    if (exact->nclass > 1) return aw_set_error(AW_EUNSUPPORTED, "the surrogate has no baseline-class input");
    if (storage != exact->spec.storage)
        return aw_set_error(AW_EUNSUPPORTED, "surrogate tables use the exact set's storage (%d), asked %d",
                            exact->spec.storage, storage);
    int rc = set_dev(s->device);
    if (rc) return rc;
    aw_kernel_set *k = new aw_kernel_set();
    k->device = exact->device;
    aw_kernel_spec sp = exact->spec;
    sp.storage = storage;
    rc = aw_kernel_set_geometry(&sp, k);
    if (rc == AW_OK) {
        k->scale = exact->scale;
        rc = aw_kernel_set_alloc(k);
    }
    if (rc == AW_OK) rc = aw_sur_tables(s, exact, k, reject_rel, bin_err, S_(stream));
    if (rc != AW_OK) {
        if (k->d_table) aw_dev_free(k->d_table);
        if (k->d_bin_support) aw_dev_free(k->d_bin_support);
        if (k->d_bin_offset) aw_dev_free(k->d_bin_offset);
        delete k;
        return rc;
    }
    *out = k;
    return k->n_rejected > 0 ? AW_EREJECTED : AW_OK;
    SUR_GUARD_END
}

int aw_surrogate_set_freq_mode(aw_surrogate *s, int32_t mode) {
    if (!s) return aw_set_error(AW_EINVAL, "surrogate is NULL");
    if (mode != AW_FREQ_BIN && mode != AW_FREQ_CHANNEL) return aw_set_error(AW_EINVAL, "frequency mode %d", mode);
    s->freq_mode = mode;
    return AW_OK;
}

int aw_surrogate_set_engine(aw_surrogate *s, int32_t engine) {
    if (!s) return aw_set_error(AW_EINVAL, "surrogate is NULL");
    if (engine != AW_ENGINE_MMA_SYNC && engine != AW_ENGINE_TCGEN05) return aw_set_error(AW_EINVAL, "engine %d", engine);
    s->engine = engine;
    return AW_OK;
}

}  // extern "C"

// Checks shared by the inline gridding and degridding, and the upload of the
// per-plane rejection flags and the bin centres the kernels read.
static int prepare_inline(const aw_plan *p, aw_surrogate *s, const aw_kernel_set *fallback, cudaStream_t st) {
    if (p->N != fallback->spec.N || p->OS != fallback->spec.OS || p->nbins != fallback->nbins ||
        p->bin_support != fallback->bin_support || p->npol != fallback->spec.npol)
        return aw_set_error(AW_EINVAL, "fallback kernel set geometry does not match the plan");
    if (fallback->nclass > 1) return aw_set_error(AW_EUNSUPPORTED, "the surrogate has no baseline-class input");
    int rc = set_dev(s->device);
    if (rc) return rc;
    const int nw = fallback->spec.nw, npa = fallback->spec.npa;
    if (!s->d_rejected) AW_CUDA_TRY(aw_dev_malloc(&s->d_rejected, 256));
    if (!s->d_pa) AW_CUDA_TRY(aw_dev_malloc(&s->d_pa, sizeof(double) * 256));
    std::vector<uint8_t> rej(nw, 0);
    for (int i = 0; i < nw && i < (int)s->plane_rejected.size(); ++i) rej[i] = s->plane_rejected[i];
    AW_CUDA_TRY(cudaMemcpyAsync(s->d_rejected, rej.data(), nw, cudaMemcpyHostToDevice, st));
    // [npa parallactic-angle centres][nfb beam-frequency centres]
    if (npa + fallback->spec.nfb > 256) return aw_set_error(AW_EUNSUPPORTED, "more than 256 PA + frequency bins");
    AW_CUDA_TRY(cudaMemcpyAsync(s->d_pa, fallback->pa.data(), sizeof(double) * npa, cudaMemcpyHostToDevice, st));
    AW_CUDA_TRY(cudaMemcpyAsync(s->d_pa + npa, fallback->fbin_freqs.data(), sizeof(double) * fallback->spec.nfb,
                                cudaMemcpyHostToDevice, st));
    return AW_OK;
}

extern "C" int aw_degrid_learned(aw_ctx *ctx, const aw_plan *p, aw_surrogate *s, const aw_kernel_set *fallback,
                                 const void *model, void *vis_out, void *stream) {
    SUR_GUARD_BEGIN
    if (!ctx || !p || !s || !fallback || !model || (!vis_out && p->nvis)) return aw_set_error(AW_EINVAL, "NULL argument");
    if (fallback->spec.role != AW_ROLE_DEGRID && fallback->spec.role != AW_ROLE_ADJOINT)
        return aw_set_error(AW_EINVAL, "the fallback set of degridding must have the DEGRID or ADJOINT role");
    cudaStream_t st = S_(stream);
    int rc = prepare_inline(p, s, fallback, st);
    if (rc) return rc;
    return aw_launch_grid_learned(p, s, fallback, s->d_rejected, s->d_pa, nullptr, nullptr, nullptr, model, vis_out,
                                  ctx->sm_count, st);
    SUR_GUARD_END
}

extern "C" int aw_grid_learned(aw_ctx *ctx, const aw_plan *p, aw_surrogate *s, const aw_kernel_set *fallback,
                               const void *vis, const float *weight, void *grid, aw_stats *stats, void *stream) {
    SUR_GUARD_BEGIN
    if (!ctx || !p || !s || !fallback || !grid || (!vis && p->nvis)) return aw_set_error(AW_EINVAL, "NULL argument");
    cudaStream_t st = S_(stream);
    int rc = prepare_inline(p, s, fallback, st);
    if (rc) return rc;
    rc = aw_launch_grid_learned(p, s, fallback, s->d_rejected, s->d_pa, vis, weight, grid, nullptr, nullptr,
                                ctx->sm_count, st);
    if (rc) return rc;
    if (stats) {
        double ws = 0;
        unsigned long long nb = 0;
        AW_CUDA_TRY(cudaMemcpyAsync(&ws, p->d_wsum, sizeof(double), cudaMemcpyDeviceToHost, st));
        AW_CUDA_TRY(cudaMemcpyAsync(&nb, p->d_nonfinite, sizeof(nb), cudaMemcpyDeviceToHost, st));
        AW_CUDA_TRY(cudaStreamSynchronize(st));
        stats->n_nonfinite = (int64_t)nb;
        stats->n_gridded = p->nvalid - (int64_t)nb;
        stats->n_outside = p->n_outside;
        stats->n_flagged = p->n_flagged;
        stats->weight_sum = ws;
    }
    return AW_OK;
    SUR_GUARD_END
}
