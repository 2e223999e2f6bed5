// mosaic_gamma_noalloc: the Eq. 1 mosaic weighting for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: host code inside a
// framework whose caching allocator already owns the device memory (a second
// allocator on the same GPU fragments it and can fail the framework's own
// requests), and real-time pipelines that forbid allocation after start-up
// (cudaMalloc can synchronise the device and take unbounded time).
// mosaic_gamma needs an aw_ctx, and aw_create allocates.  This
// variant takes no context: its only scratch is the file-scope array below,
// which every GPU that loads the library holds until the process exits.
//
// The reduction is deterministic and needs no zeroing: pass 1 writes one
// partial maximum per block into scratch[0 .. nblocks), pass 2 (one block)
// reduces exactly those slots into scratch[GAMMA_NOALLOC_BLOCKS], and pass 3
// reads that slot.  Every slot a later pass reads was written earlier in the
// same call, so the contents left by an earlier call never matter.  All calls
// share the one array: calls whose work overlaps on the GPU (different streams,
// or several host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "aw_internal.h"

#define GAMMA_NOALLOC_THREADS 256
#define GAMMA_NOALLOC_ITEMS 16
#define GAMMA_NOALLOC_BLOCKS 4096   // => at most 4096 * 256 * 16 = 4096^2 pixels

static __device__ __align__(256) float g_gamma_scratch[GAMMA_NOALLOC_BLOCKS + 1];

namespace {

constexpr int64_t kPixelsPerBlock = (int64_t)GAMMA_NOALLOC_THREADS * GAMMA_NOALLOC_ITEMS;

__global__ void noalloc_partial_max(const float *B, int nfield, int64_t npix, float *scratch) {
    __shared__ float wmax[GAMMA_NOALLOC_THREADS / 32];
    float m = 0.f;
    const int64_t base = (int64_t)blockIdx.x * kPixelsPerBlock;
    for (int i = 0; i < GAMMA_NOALLOC_ITEMS; ++i) {
        const int64_t p = base + (int64_t)i * GAMMA_NOALLOC_THREADS + threadIdx.x;
        if (p < npix) {
            float s = 0.f;
            for (int f = 0; f < nfield; ++f) {
                const float b = B[(int64_t)f * npix + p];
                s = fmaf(b, b, s);
            }
            m = fmaxf(m, sqrtf(s));
        }
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < GAMMA_NOALLOC_THREADS / 32; ++w) t = fmaxf(t, wmax[w]);
        scratch[blockIdx.x] = t;   // every block writes its slot
    }
}

__global__ void noalloc_final_max(int nblocks, float *scratch) {
    __shared__ float wmax[GAMMA_NOALLOC_THREADS / 32];
    float m = 0.f;
    for (int i = threadIdx.x; i < nblocks; i += GAMMA_NOALLOC_THREADS) m = fmaxf(m, scratch[i]);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < GAMMA_NOALLOC_THREADS / 32; ++w) t = fmaxf(t, wmax[w]);
        scratch[GAMMA_NOALLOC_BLOCKS] = t;
    }
}

__global__ void noalloc_apply(const float *B, int nfield, int64_t npix, const float *scratch, float eps,
                              float *gamma) {
    const float mx = scratch[GAMMA_NOALLOC_BLOCKS];
    const int64_t base = (int64_t)blockIdx.x * kPixelsPerBlock;
    for (int i = 0; i < GAMMA_NOALLOC_ITEMS; ++i) {
        const int64_t p = base + (int64_t)i * GAMMA_NOALLOC_THREADS + threadIdx.x;
        if (p >= npix) continue;
        float s = 0.f;
        for (int f = 0; f < nfield; ++f) {
            const float b = B[(int64_t)f * npix + p];
            s = fmaf(b, b, s);
        }
        const float pbp = (mx > 0.f) ? sqrtf(s) / mx : 0.f;
        const float wc = (s > 0.f) ? 1.0f / s : 0.f;
        gamma[p] = (pbp < eps || s == 0.f) ? 0.f : pbp * wc;
    }
}

// Device address of g_gamma_scratch, looked up with the device current (in
// host code the symbol itself is only a host-side stand-in).  A module is
// loaded per CUDA context, and a context torn down (cudaDeviceReset) and made
// again may place the array elsewhere, so the cached address is keyed on the
// identity of the current context (cuCtxGetId, unique for the life of the
// process), not on the device index: the first call in each new context looks
// the address up again.
typedef int (*ctx_get_current_fn)(void **);
typedef int (*ctx_get_id_fn)(void *, unsigned long long *);

struct ScratchSlot {
    unsigned long long ctx_id = 0;
    float *addr = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
ScratchSlot g_slot[kMaxDevices];
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

int current_context_id(unsigned long long *id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1{}, q2{};
        cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e1 != cudaSuccess || e2 != cudaSuccess || !f1 || !f2)
            return aw_set_error(AW_ECUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable");
        g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(f1);
        g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(f2);
    }
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return aw_set_error(AW_ECUDA, "no current CUDA context");
    if (g_ctx_get_id(ctx, id) != 0) return aw_set_error(AW_ECUDA, "cuCtxGetId failed");
    return AW_OK;
}

int scratch_address(int dev, float **out) {
    if (dev < 0 || dev >= kMaxDevices) return aw_set_error(AW_EUNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc) return rc;
    ScratchSlot &sl = g_slot[dev];
    if (!sl.addr || sl.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gamma_scratch);
        if (e != cudaSuccess)
            return aw_set_error(AW_ECUDA, "cudaGetSymbolAddress(g_gamma_scratch): %s", cudaGetErrorString(e));
        sl.addr = static_cast<float *>(p);
        sl.ctx_id = id;
    }
    *out = sl.addr;
    return AW_OK;
}

}  // namespace

extern "C" int mosaic_gamma_noalloc(const float *beams, int32_t nfield, int32_t N, float eps, float *gamma,
                                    void *stream) {
    try {
        if (!beams || !gamma) return aw_set_error(AW_EINVAL, "beams/gamma is NULL");
        if (nfield < 1 || N < 1) return aw_set_error(AW_EINVAL, "nfield=%d N=%d", nfield, N);
        const int64_t npix = (int64_t)N * N;
        const int64_t nblocks = (npix + kPixelsPerBlock - 1) / kPixelsPerBlock;
        if (nblocks > GAMMA_NOALLOC_BLOCKS)
            return aw_set_error(AW_EINVAL,
                                "mosaic_gamma_noalloc handles at most %lld pixels (4096 x 4096); got %d x %d",
                                (long long)GAMMA_NOALLOC_BLOCKS * kPixelsPerBlock, N, N);
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        // binds the device's primary context to this host thread (the context
        // identity below needs it current)
        e = cudaSetDevice(dev);
        if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
        float *scratch = nullptr;
        int rc = scratch_address(dev, &scratch);
        if (rc) return rc;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        noalloc_partial_max<<<(unsigned)nblocks, GAMMA_NOALLOC_THREADS, 0, s>>>(beams, nfield, npix, scratch);
        noalloc_final_max<<<1, GAMMA_NOALLOC_THREADS, 0, s>>>((int)nblocks, scratch);
        noalloc_apply<<<(unsigned)nblocks, GAMMA_NOALLOC_THREADS, 0, s>>>(beams, nfield, npix, scratch, eps, gamma);
        e = cudaGetLastError();
        if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "mosaic_gamma_noalloc launch: %s", cudaGetErrorString(e));
        return AW_OK;
    } catch (...) {
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");
    }
}
