// Internal state of the learned kernel surrogate (aw_mlp.cu, aw_learned.cu).
#pragma once

#include <vector>

#include "aw_internal.h"

struct aw_surrogate {
    int device = 0;
    aw_surrogate_cfg cfg{};
    std::vector<int> sizes;            // [5, H, ..., H, 2P]
    std::vector<int64_t> woff, boff;   // parameter offsets per layer
    int64_t nparam = 0;
    float *d_p = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr;  // FP32 master, Adam, grad
    __half *d_ph = nullptr;            // FP16 copy used by the inline evaluation
    int t = 0;                         // Adam step
    // work buffers
    int bcap = 0;
    std::vector<float *> work;
    float *X = nullptr, *T = nullptr, *dZ = nullptr, *dZ2 = nullptr, *dH = nullptr;
    std::vector<float *> Z, H;
    // per-w-plane rejection from the last aw_surrogate_tables call
    std::vector<uint8_t> plane_rejected;
    // device copies used by the inline evaluation
    uint8_t *d_rejected = nullptr;
    double *d_pa = nullptr;
    // offset-normalisation plane layout (host copy and device copy)
    std::vector<int32_t> norm;
    int32_t *d_norm = nullptr;
    // tensor-core engine of the inline evaluation (AW_ENGINE_*) and its error word
    int engine = AW_ENGINE_TCGEN05;
    unsigned int *d_err = nullptr;
    // frequency fed to the inline evaluation (AW_FREQ_*)
    int freq_mode = AW_FREQ_BIN;
    // training engine (AW_TRAIN_*) and the tensor-core path's work buffers
    int train_engine = AW_TRAIN_TCGEN05;
    struct aw_sur_tc *tc = nullptr;
};

// Tensor-core training (aw_mlp_tc.cu): width 128, at least 2 hidden layers.
int aw_sur_tc_supported(const aw_surrogate *s);
int aw_sur_tc_step_grad(aw_surrogate *s, const float *X, const float *T, int B, double *loss_dev, cudaStream_t st);
int aw_sur_tc_refresh(aw_surrogate *s, cudaStream_t st);
int aw_sur_tc_check(aw_surrogate *s, cudaStream_t st);
void aw_sur_tc_free(aw_surrogate *s);
// whether training and loss_grad take the tensor-core path
inline bool aw_sur_use_tc(const aw_surrogate *s) {
    return s->train_engine == AW_TRAIN_TCGEN05 && aw_sur_tc_supported(s);
}

// Inline evaluation: gridding (model == NULL) or, with model and vis_out,
// degridding (TCGEN05 engine only).
int aw_launch_grid_learned(const aw_plan *p, aw_surrogate *s, const aw_kernel_set *fallback, const uint8_t *d_rejected,
                           const double *d_pa, const void *vis, const float *weight, void *grid, const void *model,
                           void *vis_out, int sm_count, cudaStream_t st);

int aw_sur_init(aw_surrogate *s);
void aw_sur_free(aw_surrogate *s);
int aw_sur_alloc_work(aw_surrogate *s, int B);
int aw_sur_forward(aw_surrogate *s, const float *X, int B, cudaStream_t st);
int aw_sur_backward(aw_surrogate *s, const float *X, const float *T, int B, double *loss_dev, cudaStream_t st);
int aw_sur_adam(aw_surrogate *s, float lr, cudaStream_t st);
int aw_sur_sync_half(aw_surrogate *s, cudaStream_t st);
int aw_sur_train(aw_surrogate *s, const aw_kernel_set *k, const aw_train_cfg *tc, aw_train_report *rep,
                 cudaStream_t st);
int aw_sur_tables(aw_surrogate *s, const aw_kernel_set *exact, aw_kernel_set *out, float reject_rel,
                  float *bin_err_host, cudaStream_t st);
