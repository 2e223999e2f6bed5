// Internal declarations shared by the libaw translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdarg>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "aw.h"

#define AW_C_LIGHT 299792458.0

// ---------------------------------------------------------------- errors
int aw_set_error(int code, const char *fmt, ...);

#define AW_CUDA_TRY(call)                                                             \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return aw_set_error(e_ == cudaErrorMemoryAllocation ? AW_ENOMEM : AW_ECUDA, \
                                "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                                __FILE__, __LINE__);                                  \
    } while (0)

#define AW_CUFFT_TRY(call)                                                            \
    do {                                                                              \
        cufftResult r_ = (call);                                                      \
        if (r_ != CUFFT_SUCCESS)                                                      \
            return aw_set_error(r_ == CUFFT_ALLOC_FAILED ? AW_ENOMEM : AW_ECUDA,        \
                                "%s: cufft error %d (%s:%d)", #call, (int)r_,          \
                                __FILE__, __LINE__);                                  \
    } while (0)

#define AW_CHECK_LAUNCH() AW_CUDA_TRY(cudaGetLastError())

// ---------------------------------------------------------------- tracing
// An NVTX range named after the ABI function for the duration of the call
// (visible to profilers that attach; free otherwise).
struct AwTrace {
    explicit AwTrace(const char *name) { nvtxRangePushA(name); }
    ~AwTrace() { nvtxRangePop(); }
    AwTrace(const AwTrace &) = delete;
    AwTrace &operator=(const AwTrace &) = delete;
};
#define AW_TRACE() AwTrace aw_trace_(__func__)

// ---------------------------------------------------------------- device memory
// Every device buffer of the library goes through these: they count the live
// buffers and let aw_debug_fail_alloc make a chosen allocation fail.
cudaError_t aw_dev_malloc_raw(void **p, size_t bytes);
void aw_dev_free(void *p);
template <class T>
inline cudaError_t aw_dev_malloc(T **p, size_t bytes) {
    return aw_dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

// ---------------------------------------------------------------- handles
struct aw_ctx {
    int device = 0;
    int sm_count = 0;
    // cuFFT plans keyed by (rank tag, size, batch, type)
    std::map<std::tuple<int, int, int, int>, cufftHandle> fft_plans;
    // grid-correction vectors keyed by (N, W)
    std::map<std::pair<int, double>, float *> gridcorr;
    // small device scratch: [0] reduction word for mosaic_gamma
    unsigned int *d_scratch = nullptr;
    // last aw_autotune result (used by aw_plan_create when given no tune)
    bool has_tune = false;
    aw_tune tune_cache{};
};

struct aw_kernel_set {
    int device = 0;
    aw_kernel_spec spec{};          // copied; pointer members re-pointed to the vectors
    std::vector<int32_t> supports;  // per w plane
    std::vector<double> pa, fbin_freqs;
    std::vector<double> type_leak;  // [ntype][4] per-type leakage (ntype >= 2)
    int ntype = 1;                  // antenna types; baseline classes = ntype^2 if >= 2
    int nclass = 1;
    int nbins = 0;
    int P = 1;                      // npol * npol
    int max_support = 0;
    std::vector<int32_t> bin_support;
    std::vector<int64_t> bin_offset;  // element offset of each bin (complex elements)
    int64_t total_elems = 0;
    int elem_bytes = 8;
    // complex values per 16-byte chunk of the table layout (see aw_tab_index)
    int ce = 1;
    void *d_table = nullptr;
    int32_t *d_bin_support = nullptr;
    int64_t *d_bin_offset = nullptr;
    int n_rejected = 0;
    // tables hold K * scale (a power of two; != 1 only for FP16 storage, to keep
    // the kernel values inside the FP16 normal range)
    float scale = 1.0f;
};

// One sorted visibility: 16 bytes.
struct __align__(16) aw_rec {
    uint32_t orig;   // caller index
    uint16_t x0, y0; // first footprint cell
    uint16_t bin;
    uint8_t fx, fy;  // fine offsets
    uint8_t flip;
    uint8_t pad0;
    uint16_t pad1;
};
static_assert(sizeof(aw_rec) == 16, "aw_rec must be 16 bytes");

struct aw_plan {
    int device = 0;
    int64_t nvis = 0, nvalid = 0, n_outside = 0, n_flagged = 0, nitems = 0;
    int N = 0, OS = 0, npol = 1, nbins = 0, nw = 1, npa = 1, nfb = 1;
    int ntype = 1;                  // baseline classes are ntype^2 when ntype >= 2
    aw_tune tune{};
    double mean_taps = 0;
    aw_rec *d_rec = nullptr;        // [nvis] sorted (valid first) by (bin, tile, position)
    int4 *d_items = nullptr;        // [nitems] {start, count, bin, 0}
    // degridding order: the valid visibilities by (bin, super-tile, oversampled
    // offset, position), cut into items of at most AW_DG_CHUNK visibilities
    aw_rec *d_rec_dg = nullptr;     // [nvalid]
    int4 *d_items_dg = nullptr;     // [nitems_dg] {start, count, bin, 0}
    int64_t nitems_dg = 0;
    int dg_tile = 1024;
    int32_t *d_plane_support = nullptr;  // [nw] support per w plane
    std::vector<int32_t> bin_support;
    // grid-time statistics (device): [0] weight sum (double), [1] non-finite count
    double *d_wsum = nullptr;
    unsigned long long *d_nonfinite = nullptr;
    unsigned int *d_counter = nullptr;  // persistent work-queue head
    // AW_GRID_HYBRID: the gridding items of the low w planes (TILES) and the
    // degridding items of the others (OFFSETS), and the second stream the
    // OFFSETS part runs on (fork and join through the two events)
    int4 *d_items_ht = nullptr;
    int64_t nitems_ht = 0;
    int4 *d_items_ho = nullptr;
    int64_t nitems_ho = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // AW_GRID_REGION: the valid visibilities of the bins whose support fits a
    // shared-memory region, by (bin, region tile, oversampled offset,
    // position), cut into items {start, count, bin, tile}; one item list per
    // support (each launched with its own CTA size).  The other bins' degridding
    // items (d_items_ho) take the OFFSETS schedule on the second stream.
    aw_rec *d_rec_rg = nullptr;
    int64_t nreg = 0;
    struct RegionClass {
        int S = 0, T = 0, BT = 0;
        int4 *d_items = nullptr;
        int64_t n = 0;
    };
    std::vector<RegionClass> rclasses;
    unsigned int *d_rcounter = nullptr;   // [AW_RG_MAXCLASS] work-queue heads
    // coordinate inputs kept for aw_plan_coords
    aw_vis_desc vis{};
    double uscale = 0, half = 0, winv = 0;
    // graphs of aw_grid_batched for the last two argument sets (double-buffered
    // callers alternate between two), least recently used replaced first
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const void *vis = nullptr, *weight = nullptr, *grid = nullptr, *kset = nullptr;
        cudaStream_t stream = nullptr;
        uint64_t used = 0;
    };
    GraphSlot gslots[2];
    uint64_t gclock = 0;
    void drop_graphs() {
        for (auto &g : gslots) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = GraphSlot{};
        }
    }
};

// REGION gridding: largest region side (cells) held in shared memory, and the
// most distinct supports (item lists) a plan launches.
#ifndef AW_RG_RMAX_CELLS
#define AW_RG_RMAX_CELLS 56
#endif
constexpr int AW_RG_RMAX = AW_RG_RMAX_CELLS;
constexpr int AW_RG_MAXCLASS = 64;
constexpr int AW_RG_MAXV = 1024;   // visibilities per region work item

// Visibilities per degridding work item: 8 warps x 4 visibilities.
constexpr int AW_DG_VB = 4;
constexpr int AW_DG_CHUNK = 8 * AW_DG_VB;

// ---------------------------------------------------------------- table layout
// Inside one (bin, fy, fx) block of L = S*S taps, the P Mueller values of a tap
// are split into 16-byte chunks of `ce` complex values (ce = 2 for FP32, 4 for
// 16-bit storage, or P if P is smaller) and stored chunk-major, tap-minor:
// index(tap, m) = ((m / ce) * L + tap) * ce + m % ce.  Threads that handle
// consecutive taps then read consecutive 16-byte words (coalesced loads).
__host__ __device__ inline int64_t aw_tab_index(int ce, int64_t L, int64_t tap, int m) {
    return ((int64_t)(m / ce) * L + tap) * ce + (m % ce);
}

// ---------------------------------------------------------------- helpers
int aw_ctx_fft_plan(aw_ctx *ctx, int rank_tag, int n, int batch, cufftType type, cufftHandle *out);
int aw_ctx_gridcorr(aw_ctx *ctx, int N, double W, float **out);

// PSWF taper psi(x), psi(0) = 1, from the Legendre eigen-expansion (host).
struct aw_pswf {
    std::vector<double> beta;  // coefficients of Pbar_{2k}
    double norm = 1.0;         // 1 / psi_unnormalised(0)
    double eval(double x) const;
};
aw_pswf aw_pswf_make(double c, int nterms = 48);

// Exclusive scan of uint32 (n up to 2^31) with caller scratch from aw_scan_scratch_bytes.
size_t aw_scan_scratch_bytes(int64_t n);
int aw_exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, void *scratch,
                          cudaStream_t s);

// Grid / degrid launchers (aw_grid.cu).
struct aw_grid_launch {
    const aw_plan *plan;
    const aw_kernel_set *kset;
    const void *vis;
    const float *weight;
    void *grid;
    bool persistent;
    int ctas;
    cudaStream_t stream;
    // one schedule over a subset of its items (the parts of AW_GRID_HYBRID);
    // mode < 0: the plan's own schedule over all its items
    int mode = -1;
    const int4 *items = nullptr;
    int64_t nitems = 0;
};
int aw_launch_grid(const aw_grid_launch &L);
// REGION schedule (aw_grid_region.cu): region tile side for support S (0: the
// support does not fit a region), CTA size for support S, and the launch of
// every support's item list on stream s.
int aw_region_tile(int S, int npol);
int aw_region_rows(int S);
int aw_region_threads(int S, int npol);
int aw_launch_grid_region(const aw_plan *p, const aw_kernel_set *k, const void *vis, const float *weight, void *grid,
                          cudaStream_t s);
int aw_region_bounds_status(unsigned int *v, int reset);
// cum[q] = share of the plan's visibility-taps (sum of S^2) in w planes < q, q = 0..nw
int aw_plan_plane_taps(const aw_plan *plan, std::vector<double> &cum, cudaStream_t s);
int aw_launch_degrid(const aw_plan *plan, const aw_kernel_set *kset, const void *grid,
                     void *vis_out, cudaStream_t stream, const void *sub_from = nullptr);
int aw_fft_to_image_impl(aw_ctx *ctx, int N, int npol, double W, void *grid, double weight_sum,
                         float *image, cudaStream_t s);
int aw_image_to_grid_impl(aw_ctx *ctx, int N, int npol, double W, const float *image, void *grid,
                          cudaStream_t s);

// Storage conversion (aw_synth.cu).
int aw_export_table(const void *src, float2 *dst, int64_t nblocks, int L, int P, int ce, int storage,
                    float inv_scale, cudaStream_t s);
int aw_convert_table_scaled(const float2 *src, void *dst, int64_t nblocks, int L, int P, int ce, int storage,
                            float scale, cudaStream_t s);
int aw_table_absmax(const float2 *src, int64_t n, float *out_host, cudaStream_t s);
