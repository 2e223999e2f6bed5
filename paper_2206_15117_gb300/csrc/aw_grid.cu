// Gridding and degridding kernels: the hot path.
//
// arXiv:2206.15117 Sec. 3.2: gridding convolves every visibility onto the uv
// grid with the oversampled kernel of its bin (uv transform of the inverse
// Mueller cells); degridding gathers the model grid back with the kernels of
// the Mueller cells (Eq. 5).  Sec. 2.1: w-projection with a configurable
// number of w planes.
//
// Gridding: one CTA per work item (a run of at most `chunk` visibilities of
// one bin and one grid tile, sorted by position).  The item's visibilities
// (flipped, weighted, NaN-checked) are staged in shared memory.  Each thread
// owns one residue class (a, b) of grid cells modulo the support S: for any
// visibility exactly one cell of its S x S footprint is in that class.  The
// thread accumulates that cell's contribution in registers while consecutive
// visibilities keep hitting the same cell and adds it to HBM with one vector
// atomic per plane when the cell changes.  The 4x4 Mueller kernel of a tap
// (16 complex values, 128 B in FP32) is read with 128-bit loads.
//
// Degridding: one warp per visibility; lanes stride over the S x S taps,
// each tap a (npol x npol) complex kernel times npol grid values, then a
// warp-shuffle reduction.
#include <algorithm>

#include "aw_internal.h"

namespace {

template <int ST>
struct KTraits;
template <>
struct KTraits<AW_STORAGE_FP32> {
    using T = float2;
};
template <>
struct KTraits<AW_STORAGE_BF16> {
    using T = __nv_bfloat162;
};
template <>
struct KTraits<AW_STORAGE_FP16> {
    using T = __half2;
};

// Load the P Mueller values of tap `tap` of a (bin, fy, fx) block of L taps
// that starts at complex element `base_idx`, in the chunked layout of
// aw_tab_index: chunk c of every tap is contiguous over taps, so lanes that
// handle consecutive taps issue coalesced 16-byte loads.
template <int ST, int P>
__device__ __forceinline__ void load_k(const void *base, int64_t base_idx, int L, int tap, float2 (&k)[P]) {
    if constexpr (ST == AW_STORAGE_FP32) {
        const float2 *p = reinterpret_cast<const float2 *>(base) + base_idx;
        if constexpr (P % 2 == 0) {
#pragma unroll
            for (int c = 0; c < P / 2; ++c) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(p + 2 * ((int64_t)c * L + tap)));
                k[2 * c] = make_float2(v.x, v.y);
                k[2 * c + 1] = make_float2(v.z, v.w);
            }
        } else {
            k[0] = __ldg(p + tap);
        }
    } else {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(base) + base_idx;
        if constexpr (P % 4 == 0) {
#pragma unroll
            for (int c = 0; c < P / 4; ++c) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + 4 * ((int64_t)c * L + tap)));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if constexpr (ST == AW_STORAGE_BF16) {
                        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[j]);
                        k[4 * c + j] = __bfloat1622float2(h);
                    } else {
                        __half2 h = *reinterpret_cast<const __half2 *>(&w[j]);
                        k[4 * c + j] = __half22float2(h);
                    }
                }
            }
        } else {
            const uint32_t w = __ldg(p + tap);
            if constexpr (ST == AW_STORAGE_BF16) {
                __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w);
                k[0] = __bfloat1622float2(h);
            } else {
                __half2 h = *reinterpret_cast<const __half2 *>(&w);
                k[0] = __half22float2(h);
            }
        }
    }
}

__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

struct GridArgs {
    const aw_rec *rec;
    const int4 *items;
    int64_t nitems;
    const void *ktab;
    const int64_t *bin_offset;
    const int32_t *bin_support;
    const float2 *vis;
    const float *weight;
    float2 *grid;
    int N, OS;
    int chunk;
    double *wsum;
    unsigned long long *nonfinite;
    unsigned int *counter;   // persistent queue head
    float inv_scale;         // 1 / table scale
};

template <int NPOL>
struct SmemLayout {
    // per staged visibility: int4 {x0 | y0 << 16, (x0 mod S) | (y0 mod S) << 16,
    // kernel block offset, 0} and NPOL weighted complex values
    static __host__ __device__ size_t bytes(int chunk) {
        return (size_t)chunk * (sizeof(int4) + NPOL * sizeof(float2));
    }
};

template <int NPOL, int ST>
__device__ __forceinline__ void grid_one_item(const GridArgs &a, int item, char *smem, double *red) {
    constexpr int P = NPOL * NPOL;
    const int4 it = a.items[item];
    const int start = it.x, count = it.y, bin = it.z;
    const int S = a.bin_support[bin];
    const int64_t tab0 = a.bin_offset[bin];
    int4 *s_meta = reinterpret_cast<int4 *>(smem);
    float2 *s_v = reinterpret_cast<float2 *>(s_meta + a.chunk);
    // ---- stage the item's visibilities
    double wloc = 0.0;
    unsigned long long nbad = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const aw_rec r = a.rec[start + i];
        float2 v[NPOL];
        float w[NPOL];
        bool bad = false;
#pragma unroll
        for (int c = 0; c < NPOL; ++c) {
            v[c] = a.vis[(int64_t)r.orig * NPOL + c];
            w[c] = a.weight ? a.weight[(int64_t)r.orig * NPOL + c] : 1.0f;
            bad |= !isfinite(v[c].x) || !isfinite(v[c].y) || !isfinite(w[c]);
        }
        if (r.flip) {
#pragma unroll
            for (int c = 0; c < NPOL; ++c) v[c].y = -v[c].y;
            if (NPOL == 4) {
                float2 t = v[1]; v[1] = v[2]; v[2] = t;
                float tw = w[1]; w[1] = w[2]; w[2] = tw;
            }
        }
        if (bad) {
            nbad++;
#pragma unroll
            for (int c = 0; c < NPOL; ++c) { v[c] = make_float2(0.f, 0.f); w[c] = 0.f; }
        }
        double wm = 0.0;
#pragma unroll
        for (int c = 0; c < NPOL; ++c) {
            wm += (double)w[c];
            const float ws = w[c] * a.inv_scale;
            s_v[i * NPOL + c] = make_float2(ws * v[c].x, ws * v[c].y);
        }
        wloc += wm / NPOL;
        s_meta[i] = make_int4((int)r.x0 | ((int)r.y0 << 16), ((int)r.x0 % S) | (((int)r.y0 % S) << 16),
                              ((int)r.fy * a.OS + (int)r.fx) * S * S * P, 0);
    }
    // block reduction of the weight sum (double) and the non-finite count
    for (int o = 16; o; o >>= 1) {
        wloc += __shfl_xor_sync(0xffffffffu, wloc, o);
        nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = wloc;
    if (nbad && lane == 0) atomicAdd(a.nonfinite, nbad);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(a.wsum, t);
    }
    // ---- owner-class accumulation
    const int L = S * S;
    const int NT = blockDim.x;
    const int G = (L >= NT) ? 1 : min(NT / L, 32);
    const int active = (L >= NT) ? NT : G * L;
    if ((int)threadIdx.x < active) {
        const int g = (L >= NT) ? 0 : (int)threadIdx.x / L;
        const int q0 = (L >= NT) ? (int)threadIdx.x : (int)threadIdx.x % L;
        const int qstep = (L >= NT) ? NT : L;
        for (int q = q0; q < L; q += qstep) {
            const int ca = q % S, cb = q / S;
            int cur = -1;
            float2 acc[NPOL];
#pragma unroll
            for (int s = 0; s < NPOL; ++s) acc[s] = make_float2(0.f, 0.f);
            for (int i = g; i < count; i += G) {
                const int4 meta = s_meta[i];
                const int pos = meta.x;
                const int md = meta.y;
                int jx = ca - (md & 0xffff);
                jx += (jx < 0) ? S : 0;
                int jy = cb - (md >> 16);
                jy += (jy < 0) ? S : 0;
                const int gx = (pos & 0xffff) + jx;
                const int gy = (pos >> 16) + jy;
                const int key = gx | (gy << 16);
                if (key != cur) {
                    if (cur >= 0) {
                        const int cx = cur & 0xffff, cy = cur >> 16;
#pragma unroll
                        for (int s = 0; s < NPOL; ++s)
                            atomicAdd(a.grid + ((int64_t)s * a.N + cy) * a.N + cx, acc[s]);
                    }
                    cur = key;
#pragma unroll
                    for (int s = 0; s < NPOL; ++s) acc[s] = make_float2(0.f, 0.f);
                }
                float2 k[P];
                load_k<ST, P>(a.ktab, tab0 + meta.z, L, jy * S + jx, k);
                float2 v[NPOL];
                if constexpr (NPOL == 4) {
                    const float4 v01 = reinterpret_cast<const float4 *>(s_v)[2 * i];
                    const float4 v23 = reinterpret_cast<const float4 *>(s_v)[2 * i + 1];
                    v[0] = make_float2(v01.x, v01.y); v[1] = make_float2(v01.z, v01.w);
                    v[2] = make_float2(v23.x, v23.y); v[3] = make_float2(v23.z, v23.w);
                } else {
                    v[0] = s_v[i];
                }
#pragma unroll
                for (int s = 0; s < NPOL; ++s)
#pragma unroll
                    for (int c = 0; c < NPOL; ++c) cmac(acc[s], k[s * NPOL + c], v[c]);
            }
            if (cur >= 0) {
                const int cx = cur & 0xffff, cy = cur >> 16;
#pragma unroll
                for (int s = 0; s < NPOL; ++s)
                    atomicAdd(a.grid + ((int64_t)s * a.N + cy) * a.N + cx, acc[s]);
            }
        }
    }
}

template <int NPOL, int ST>
__global__ void __launch_bounds__(256) grid_items_kernel(GridArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ double red[8];
    grid_one_item<NPOL, ST>(a, blockIdx.x, smem, red);
}

// Persistent form: CTAs pull items from a device queue until it is empty.
template <int NPOL, int ST>
__global__ void __launch_bounds__(256, 5) grid_persistent_kernel(GridArgs a) {
    extern __shared__ __align__(16) char smem[];
    __shared__ double red[8];
    __shared__ int next;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) next = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = next;
        if (item >= a.nitems) break;
        grid_one_item<NPOL, ST>(a, item, smem, red);
    }
}

struct DegridArgs {
    const aw_rec *rec;
    int64_t nvis, nvalid;
    const void *ktab;
    const int64_t *bin_offset;
    const int32_t *bin_support;
    const float2 *grid;
    float2 *vis_out;
    int N, OS;
    float inv_scale;
};

template <int NPOL, int ST>
__global__ void __launch_bounds__(256, 5) degrid_warp_kernel(DegridArgs a) {
    constexpr int P = NPOL * NPOL;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < a.nvis; i += warps) {
        const aw_rec r = a.rec[i];
        if (i >= a.nvalid) {
            if (lane < NPOL) a.vis_out[(int64_t)r.orig * NPOL + lane] = make_float2(0.f, 0.f);
            continue;
        }
        const int S = a.bin_support[r.bin];
        const int L = S * S;
        const int64_t kbase = a.bin_offset[r.bin] + (int64_t)(r.fy * a.OS + r.fx) * L * P;  // block start
        const float2 *g0 = a.grid + (int64_t)r.y0 * a.N + r.x0;
        const int64_t plane = (int64_t)a.N * a.N;
        float2 acc[NPOL];
#pragma unroll
        for (int c = 0; c < NPOL; ++c) acc[c] = make_float2(0.f, 0.f);
        int jy = lane / S, jx = lane - jy * S;
        for (int t = lane; t < L; t += 32) {
            float2 k[P];
            load_k<ST, P>(a.ktab, kbase, L, t, k);
            const float2 *gp = g0 + (int64_t)jy * a.N + jx;
            float2 gv[NPOL];
#pragma unroll
            for (int s = 0; s < NPOL; ++s) gv[s] = __ldg(gp + s * plane);
#pragma unroll
            for (int c = 0; c < NPOL; ++c)
#pragma unroll
                for (int s = 0; s < NPOL; ++s) cmac(acc[c], k[c * NPOL + s], gv[s]);
            jx += 32;
            while (jx >= S) { jx -= S; ++jy; }
        }
#pragma unroll
        for (int c = 0; c < NPOL; ++c)
            for (int o = 16; o; o >>= 1) {
                acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, o);
                acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, o);
            }
        if (lane == 0) {
            float2 out[NPOL];
#pragma unroll
            for (int c = 0; c < NPOL; ++c) out[c] = make_float2(acc[c].x * a.inv_scale, acc[c].y * a.inv_scale);
            if (r.flip) {
#pragma unroll
                for (int c = 0; c < NPOL; ++c) out[c].y = -out[c].y;
                if (NPOL == 4) { float2 t = out[1]; out[1] = out[2]; out[2] = t; }
            }
            float2 *dst = a.vis_out + (int64_t)r.orig * NPOL;
            if constexpr (NPOL == 4) {
                reinterpret_cast<float4 *>(dst)[0] = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
                reinterpret_cast<float4 *>(dst)[1] = make_float4(out[2].x, out[2].y, out[3].x, out[3].y);
            } else {
                dst[0] = out[0];
            }
        }
    }
}

template <int NPOL, int ST>
int launch_grid_t(const aw_grid_launch &L, const GridArgs &a) {
    const size_t smem = SmemLayout<NPOL>::bytes(a.chunk);
    auto kern = L.persistent ? grid_persistent_kernel<NPOL, ST> : grid_items_kernel<NPOL, ST>;
    AW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (L.persistent) {
        grid_persistent_kernel<NPOL, ST><<<L.ctas, 256, smem, L.stream>>>(a);
    } else {
        grid_items_kernel<NPOL, ST><<<(unsigned)a.nitems, 256, smem, L.stream>>>(a);
    }
    AW_CHECK_LAUNCH();
    return AW_OK;
}

template <int NPOL, int ST>
int launch_degrid_t(const DegridArgs &a, int sm_count, cudaStream_t s) {
    int64_t blocks = (a.nvis + 7) / 8;
    const int64_t cap = (int64_t)sm_count * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    degrid_warp_kernel<NPOL, ST><<<(unsigned)blocks, 256, 0, s>>>(a);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

}  // namespace

int aw_launch_grid(const aw_grid_launch &L) {
    const aw_plan *p = L.plan;
    const aw_kernel_set *k = L.kset;
    if (p->nitems == 0) return AW_OK;
    GridArgs a;
    a.rec = p->d_rec;
    a.items = p->d_items;
    a.nitems = p->nitems;
    a.ktab = k->d_table;
    a.bin_offset = k->d_bin_offset;
    a.bin_support = k->d_bin_support;
    a.vis = reinterpret_cast<const float2 *>(L.vis);
    a.weight = L.weight;
    a.grid = reinterpret_cast<float2 *>(L.grid);
    a.N = p->N;
    a.OS = p->OS;
    a.chunk = p->tune.chunk;
    a.wsum = p->d_wsum;
    a.nonfinite = p->d_nonfinite;
    a.counter = p->d_counter;
    a.inv_scale = 1.0f / k->scale;
    const int st = k->spec.storage;
    if (p->npol == 1) {
        if (st == AW_STORAGE_FP32) return launch_grid_t<1, AW_STORAGE_FP32>(L, a);
        if (st == AW_STORAGE_BF16) return launch_grid_t<1, AW_STORAGE_BF16>(L, a);
        return launch_grid_t<1, AW_STORAGE_FP16>(L, a);
    }
    if (st == AW_STORAGE_FP32) return launch_grid_t<4, AW_STORAGE_FP32>(L, a);
    if (st == AW_STORAGE_BF16) return launch_grid_t<4, AW_STORAGE_BF16>(L, a);
    return launch_grid_t<4, AW_STORAGE_FP16>(L, a);
}

int aw_launch_degrid(const aw_plan *p, const aw_kernel_set *k, const void *grid, void *vis_out,
                     cudaStream_t s) {
    if (p->nvis == 0) return AW_OK;
    DegridArgs a;
    a.rec = p->d_rec;
    a.nvis = p->nvis;
    a.nvalid = p->nvalid;
    a.ktab = k->d_table;
    a.bin_offset = k->d_bin_offset;
    a.bin_support = k->d_bin_support;
    a.grid = reinterpret_cast<const float2 *>(grid);
    a.vis_out = reinterpret_cast<float2 *>(vis_out);
    a.N = p->N;
    a.OS = p->OS;
    a.inv_scale = 1.0f / k->scale;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int st = k->spec.storage;
    if (p->npol == 1) {
        if (st == AW_STORAGE_FP32) return launch_degrid_t<1, AW_STORAGE_FP32>(a, sms, s);
        if (st == AW_STORAGE_BF16) return launch_degrid_t<1, AW_STORAGE_BF16>(a, sms, s);
        return launch_degrid_t<1, AW_STORAGE_FP16>(a, sms, s);
    }
    if (st == AW_STORAGE_FP32) return launch_degrid_t<4, AW_STORAGE_FP32>(a, sms, s);
    if (st == AW_STORAGE_BF16) return launch_degrid_t<4, AW_STORAGE_BF16>(a, sms, s);
    return launch_degrid_t<4, AW_STORAGE_FP16>(a, sms, s);
}
