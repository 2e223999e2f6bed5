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
// Degridding: visibilities grouped by (bin, grid super-tile, oversampled
// offset) share one kernel block; a CTA stages that block in shared memory
// and applies it to up to 32 visibilities, each tap an (npol x npol) complex
// kernel times npol grid values read from the super-tile (L2-resident).
#include <algorithm>

#include "aw_internal.h"

// Debug builds with -DAW_BOUNDS_CHECK check every grid, table, shared-memory,
// record and output index of the kernels in this file: a bad index records a
// code in a device status word (the first one wins) and the access is
// skipped.  Normal builds compile the checks away.
#ifdef AW_BOUNDS_CHECK
__device__ unsigned int g_bounds_status;
#endif

namespace {

#ifdef AW_BOUNDS_CHECK
__device__ __forceinline__ bool bounds_ok(bool ok, unsigned int code) {
    if (!ok) atomicCAS(&g_bounds_status, 0u, code);
    return ok;
}
#define AW_BOK(cond, code) bounds_ok((cond), (code))
#else
#define AW_BOK(cond, code) true
#endif

// codes of the bounds checks
enum : unsigned int {
    BC_T_GRID = 1, BC_T_TAB, BC_T_SMEM, BC_T_REC,        // tile schedule
    BC_O_GRID = 5, BC_O_TAB, BC_O_SMEM, BC_O_REC,        // offset schedule
    BC_D_SRC = 9, BC_D_DST, BC_D_GRID, BC_D_OUT, BC_D_REC  // degridding
};

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
    int64_t nvis, nvalid, tab_elems;  // extents for the bounds checks
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
        if (!AW_BOK(i < a.chunk && start + i < a.nvalid, BC_T_SMEM)) continue;
        const aw_rec r = a.rec[start + i];
        if (!AW_BOK(r.orig < a.nvis, BC_T_REC)) continue;
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
                if (!AW_BOK(i < a.chunk, BC_T_SMEM)) break;
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
                        if (AW_BOK(cx < a.N && cy < a.N, BC_T_GRID))
#pragma unroll
                            for (int s = 0; s < NPOL; ++s)
                                atomicAdd(a.grid + ((int64_t)s * a.N + cy) * a.N + cx, acc[s]);
                    }
                    cur = key;
#pragma unroll
                    for (int s = 0; s < NPOL; ++s) acc[s] = make_float2(0.f, 0.f);
                }
                float2 k[P];
                if (!AW_BOK(meta.z >= 0 && tab0 + meta.z + (int64_t)P * L <= a.tab_elems && jy * S + jx < L,
                            BC_T_TAB))
                    continue;
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
                if (AW_BOK(cx < a.N && cy < a.N, BC_T_GRID))
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

// Offset-grouped form of gridding, over the degridding items (visibilities
// that share the bin and the oversampled offset, hence one kernel block).
// A task is one tap t of the block and one residue class p of the item's
// visibilities modulo nsplit: it loads the P Mueller values of tap t once and
// applies them to every visibility of its class, adding each product to the
// grid with one vector atomic per plane.  nsplit makes the task count a
// multiple of the CTA size.  Weight-sum and non-finite statistics are kept
// per thread over all its items and reduced once at the end.
struct GridOffArgs {
    const aw_rec *rec_dg;
    const int4 *items;
    int64_t nitems;
    const void *ktab;
    const int64_t *bin_offset;
    const int32_t *bin_support;
    const float2 *vis;
    const float *weight;
    float2 *grid;
    int N, OS;
    double *wsum;
    unsigned long long *nonfinite;
    float inv_scale;
    int64_t nvis, nvalid, tab_elems;  // extents for the bounds checks
};

__host__ __device__ inline int gcd_i(int a, int b) {
    while (b) { const int t = a % b; a = b; b = t; }
    return a;
}

template <int NPOL, int ST>
__global__ void __launch_bounds__(256) grid_offset_kernel(GridOffArgs a) {
    constexpr int P = NPOL * NPOL;
    __shared__ __align__(16) float2 s_v[AW_DG_CHUNK * NPOL];
    __shared__ int2 s_pos[AW_DG_CHUNK];
    __shared__ double red[8];
    __shared__ unsigned long long redn[8];
    const int64_t plane = (int64_t)a.N * a.N;
    double wloc = 0.0;
    unsigned long long nbad = 0;
    for (int64_t item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int4 it = a.items[item];
        const int start = it.x, count = it.y, bin = it.z;
        const int S = a.bin_support[bin];
        const int L = S * S;
        const float invS = 1.0f / (float)S;
        __syncthreads();  // the previous item has finished with s_v / s_pos
        if ((int)threadIdx.x < count && AW_BOK(count <= AW_DG_CHUNK && start + (int)threadIdx.x < a.nvalid, BC_O_SMEM)) {
            const aw_rec r = a.rec_dg[start + threadIdx.x];
            // (checked builds: a bad record reads visibility 0 instead)
            const int64_t orig = AW_BOK(r.orig < a.nvis, BC_O_REC) ? (int64_t)r.orig : 0;
            float2 v[NPOL];
            float w[NPOL];
            bool bad = false;
#pragma unroll
            for (int c = 0; c < NPOL; ++c) {
                v[c] = a.vis[orig * NPOL + c];
                w[c] = a.weight ? a.weight[orig * NPOL + c] : 1.0f;
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
                s_v[threadIdx.x * NPOL + c] = make_float2(ws * v[c].x, ws * v[c].y);
            }
            wloc += wm / NPOL;
            s_pos[threadIdx.x] = make_int2(r.x0, r.y0);
        }
        __syncthreads();
        const aw_rec r0 = a.rec_dg[start];
        const int64_t kbase = a.bin_offset[bin] + (int64_t)(r0.fy * a.OS + r0.fx) * L * P;
        const int nsplit = min(256 / gcd_i(L, 256), 8);
        const int ntask = L * nsplit;
        for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
            const int p = task / L, t = task - p * L;  // lanes on consecutive taps
            const int jy = (int)(((float)t + 0.5f) * invS);
            const int jx = t - jy * S;
            float2 k[P];
            if (!AW_BOK(kbase >= 0 && kbase + (int64_t)P * L <= a.tab_elems, BC_O_TAB)) continue;
            load_k<ST, P>(a.ktab, kbase, L, t, k);
            for (int j = p; j < count && AW_BOK(j < AW_DG_CHUNK, BC_O_SMEM); j += nsplit) {
                float2 v[NPOL];
                if constexpr (NPOL == 4) {
                    const float4 v01 = reinterpret_cast<const float4 *>(s_v)[2 * j];
                    const float4 v23 = reinterpret_cast<const float4 *>(s_v)[2 * j + 1];
                    v[0] = make_float2(v01.x, v01.y); v[1] = make_float2(v01.z, v01.w);
                    v[2] = make_float2(v23.x, v23.y); v[3] = make_float2(v23.z, v23.w);
                } else {
                    v[0] = s_v[j];
                }
                const int2 pos = s_pos[j];
                if (!AW_BOK(pos.x >= 0 && pos.y >= 0 && pos.x + jx < a.N && pos.y + jy < a.N, BC_O_GRID)) continue;
                float2 *dst = a.grid + (int64_t)(pos.y + jy) * a.N + (pos.x + jx);
#pragma unroll
                for (int s = 0; s < NPOL; ++s) {
                    float2 o = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < NPOL; ++c) cmac(o, k[s * NPOL + c], v[c]);
                    atomicAdd(dst + s * plane, o);
                }
            }
        }
    }
    // statistics: one atomic per CTA
    for (int o = 16; o; o >>= 1) {
        wloc += __shfl_xor_sync(0xffffffffu, wloc, o);
        nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[warp] = wloc; redn[warp] = nbad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tw = 0.0;
        unsigned long long tn = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tw += red[w]; tn += redn[w]; }
        atomicAdd(a.wsum, tw);
        if (tn) atomicAdd(a.nonfinite, tn);
    }
}

struct DegridArgs {
    const aw_rec *rec;       // grid order: [nvalid, nvis) are the visibilities not gridded
    const aw_rec *rec_dg;    // [nvalid] degridding order
    const int4 *items;       // [nitems] {start, count, bin, 0} over rec_dg
    int64_t nitems;
    int64_t nvis, nvalid;
    const void *ktab;
    const int64_t *bin_offset;
    const int32_t *bin_support;
    const float2 *grid;
    float2 *vis_out;
    const float2 *sub_from;  // if set: vis_out = sub_from - prediction (may alias vis_out)
    int N, OS;
    float inv_scale;
    int64_t tab_elems;       // table extent for the bounds checks
};

constexpr int DG_TS = 256;  // taps per shared-memory slab of the kernel block

// Warp sum of x[0..2H) over the 32 lanes, halving the values held at each
// step (reduce-scatter): for 2H == 32, lane l returns with the sum of x[l] in x[0].
template <int H>
__device__ __forceinline__ void reduce_scatter_step(float *x, int lane) {
    const bool up = (lane & H) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float send = up ? x[i] : x[i + H];
        const float keep = up ? x[i + H] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, H);
    }
    if constexpr (H > 1) reduce_scatter_step<H / 2>(x, lane);
}

// Kernel-table chunk geometry of one tap: NCH chunks of CB bytes each (the
// 16-byte chunks of aw_tab_index, or one element when P == 1).
template <int P, int ST>
struct TabChunks {
    static constexpr int EB = (ST == AW_STORAGE_FP32) ? 8 : 4;   // bytes per complex value
    static constexpr int CE = (P == 1) ? 1 : 16 / EB;            // complex values per chunk
    static constexpr int CB = CE * EB;                           // bytes per chunk
    static constexpr int NCH = P / CE;                           // chunks per tap
    static constexpr int SLAB_BYTES = DG_TS * NCH * CB;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <int CB>
__device__ __forceinline__ void cp_async_chunk(uint32_t dst, const void *src) {
    if constexpr (CB == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(src), "n"(CB) : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Mueller row c (values c*NPOL .. c*NPOL+NPOL-1) of tap tl from a staged slab.
template <int NPOL, int ST>
__device__ __forceinline__ void smem_krow(const char *slab, int tl, int c, float2 (&k)[NPOL]) {
    using TC = TabChunks<NPOL * NPOL, ST>;
    if constexpr (NPOL == 1) {
        if constexpr (ST == AW_STORAGE_FP32) {
            k[0] = reinterpret_cast<const float2 *>(slab)[tl];
        } else {
            const uint32_t w = reinterpret_cast<const uint32_t *>(slab)[tl];
            if constexpr (ST == AW_STORAGE_BF16) k[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
            else k[0] = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        }
    } else if constexpr (ST == AW_STORAGE_FP32) {
        // row c = chunks 2c and 2c+1 (two complex values each)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 q = reinterpret_cast<const float4 *>(slab)[(2 * c + h) * DG_TS + tl];
            k[2 * h] = make_float2(q.x, q.y);
            k[2 * h + 1] = make_float2(q.z, q.w);
        }
    } else {
        // row c = chunk c (four complex values)
        const uint4 q = reinterpret_cast<const uint4 *>(slab)[c * DG_TS + tl];
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if constexpr (ST == AW_STORAGE_BF16) k[j] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[j]));
            else k[j] = __half22float2(*reinterpret_cast<const __half2 *>(&w[j]));
        }
    }
    (void)sizeof(TC);
}

// One CTA works through the items b, b + gridDim.x, ... (up to AW_DG_CHUNK
// visibilities that share the bin and the oversampled offset (fy, fx), hence
// one kernel block of S*S taps).  The block is staged in shared memory in
// slabs of DG_TS taps, in the table's own storage format, with cp.async into
// two buffers: the next slab (of this item or the next) streams in while the
// current one is used.  The visibilities are dealt to ngp warp groups
// (v = g + ngp * j, j < AW_DG_VB); the warps of a group split the taps; lanes
// stride over taps, load the npol grid values of their taps for every
// visibility first, then apply the kernel one Mueller row at a time.  Partial
// sums (AW_DG_VB x NPOL complex per lane) are reduce-scattered over the warp
// and summed across the group's warps in shared memory.
// Stokes I: at most 64 registers, four CTAs per SM (the kernel hides the
// latency of its grid loads with resident warps).
template <int NPOL, int ST, bool SUB>
__global__ void __launch_bounds__(256, NPOL == 1 ? 4 : 2) degrid_items_kernel(DegridArgs a) {
    constexpr int P = NPOL * NPOL;
    constexpr int VB = AW_DG_VB;
    constexpr int NV = VB * NPOL * 2;  // partial sums per lane
    using TC = TabChunks<P, ST>;
    extern __shared__ __align__(16) char dsm[];
    // full-pol with 16-bit tables: each slab is widened to FP32 once, into s_f32, so
    // that the eight warps reading every tap do not each convert it again
    constexpr bool CONV = NPOL == 4 && ST != AW_STORAGE_FP32;
    using TF = TabChunks<P, AW_STORAGE_FP32>;
    char *s_f32 = dsm + 2 * TC::SLAB_BYTES;
    float *s_out = reinterpret_cast<float *>(s_f32 + (CONV ? TF::SLAB_BYTES : 0));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float2 *gplane[NPOL];
#pragma unroll
    for (int s2 = 0; s2 < NPOL; ++s2) gplane[s2] = a.grid + (int64_t)s2 * a.N * a.N;
    const char *ktab = reinterpret_cast<const char *>(a.ktab);

    // ---- an item's header: its records, support and kernel block
    struct Hdr {
        int start, count, S;
        int64_t kbase;  // complex index of the kernel block in the table
    };
    auto load_hdr = [&](int64_t item) {
        const int4 it = a.items[item];
        Hdr h;
        h.start = it.x;
        h.count = it.y;
        h.S = a.bin_support[it.z];
        const aw_rec r0 = a.rec_dg[it.x];
        h.kbase = a.bin_offset[it.z] + (int64_t)(r0.fy * a.OS + r0.fx) * h.S * h.S * P;
        return h;
    };
    // ---- staging of slab `slab` of an item into buffer b
    auto stage = [&](const Hdr &h, int slab, int b) {
        const int L = h.S * h.S;
        const int64_t kbase = h.kbase;
        const char *src = ktab + kbase * TC::EB;
        const int t0 = slab * DG_TS;
        const int ns = min(DG_TS, L - t0);
        const uint32_t dst = smem_u32(dsm) + (uint32_t)(b * TC::SLAB_BYTES);
        // a thread per tap copies the tap's NCH chunks (one pass when blockDim.x == DG_TS);
        // for each chunk index the lanes of a warp read consecutive 16-byte chunks
        for (int tl = threadIdx.x; tl < ns; tl += blockDim.x) {
            const char *s0 = src + ((int64_t)t0 + tl) * TC::CB;
#pragma unroll
            for (int c = 0; c < TC::NCH; ++c)
                if (AW_BOK(kbase >= 0 && kbase + ((int64_t)c * L + t0 + tl + 1) * TC::CE <= a.tab_elems, BC_D_SRC) &&
                    AW_BOK(tl < DG_TS, BC_D_DST))
                    cp_async_chunk<TC::CB>(dst + (uint32_t)((c * DG_TS + tl) * TC::CB), s0 + (int64_t)c * L * TC::CB);
        }
        cp_async_commit();
    };
    auto nslabs = [&](const Hdr &h) { return (h.S * h.S + DG_TS - 1) / DG_TS; };

    int64_t item = blockIdx.x;
    if (item < a.nitems) {
        // the next item's header is loaded as soon as an item starts, so that
        // its latency hides behind the item's slabs
        Hdr cur = load_hdr(item), nxt = cur;
        bool nxt_ok = item + gridDim.x < a.nitems;
        if (nxt_ok) nxt = load_hdr(item + gridDim.x);
        int slab = 0, nsl = nslabs(cur), buf = 0;
        stage(cur, 0, 0);
        // per-item state
        int start = 0, count = 0, S = 0, L = 0, ngp = 1, wpg = 8, g = 0, ph = 0;
        float invS = 1.f;
        uint32_t goff[VB];  // y0 * N + x0 (< 2^32: coordinates are 16-bit)
        bool has[VB];
        float acc[NV];
        for (;;) {
            if (slab == 0) {
                start = cur.start; count = cur.count;
                S = cur.S;
                L = S * S;
                invS = 1.0f / (float)S;
                const int need = (count + VB - 1) / VB;
                ngp = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : 8;
                wpg = 8 / ngp;
                g = warp & (ngp - 1);
                ph = warp / ngp;
#pragma unroll
                for (int j = 0; j < VB; ++j) {
                    const int v = g + ngp * j;
                    has[j] = v < count;
                    const bool inr = AW_BOK(start + (has[j] ? v : 0) < a.nvalid, BC_D_REC);
                    has[j] = has[j] && inr;
                    const aw_rec r = a.rec_dg[inr ? start + (has[j] ? v : 0) : 0];
                    goff[j] = (uint32_t)r.y0 * (uint32_t)a.N + r.x0;
                }
#pragma unroll
                for (int i = 0; i < NV; ++i) acc[i] = 0.f;
                for (int i = threadIdx.x; i < count * NPOL * 2; i += blockDim.x)
                    if (AW_BOK(i < AW_DG_CHUNK * NPOL * 2, BC_D_OUT)) s_out[i] = 0.f;
            }
            // the next (item, slab) streams into the other buffer
            const bool to_next = slab + 1 == nsl;
            const bool has_next = !to_next || nxt_ok;
            if (has_next) {
                stage(to_next ? nxt : cur, to_next ? 0 : slab + 1, buf ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const char *sl = dsm + buf * TC::SLAB_BYTES;
            const int t0 = slab * DG_TS;
            const int ns = min(DG_TS, L - t0);
            if constexpr (CONV) {
                // row c of a tap: one 16-byte chunk of four 16-bit complex values in the
                // staged slab, two chunks of two FP32 complex values in s_f32
                for (int tl = threadIdx.x; tl < ns; tl += blockDim.x) {
#pragma unroll
                    for (int c = 0; c < NPOL; ++c) {
                        float2 kr[NPOL];
                        smem_krow<NPOL, ST>(sl, tl, c, kr);
                        float4 *d = reinterpret_cast<float4 *>(s_f32);
                        d[(2 * c) * DG_TS + tl] = make_float4(kr[0].x, kr[0].y, kr[1].x, kr[1].y);
                        d[(2 * c + 1) * DG_TS + tl] = make_float4(kr[2].x, kr[2].y, kr[3].x, kr[3].y);
                    }
                }
                __syncthreads();
                sl = s_f32;
            }
            for (int tl = ph * 32 + lane; tl < ns; tl += wpg * 32) {
                const int t = t0 + tl;
                const int jy = (int)(((float)t + 0.5f) * invS);
                const uint32_t toff = (uint32_t)(jy * a.N + (t - jy * S));
                float2 gv[VB][NPOL];
#pragma unroll
                for (int j = 0; j < VB; ++j) {
#pragma unroll
                    for (int s2 = 0; s2 < NPOL; ++s2)
                        gv[j][s2] = (has[j] && AW_BOK(goff[j] + toff < (uint32_t)a.N * (uint32_t)a.N, BC_D_GRID))
                                        ? __ldg(gplane[s2] + (goff[j] + toff))
                                        : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int c = 0; c < NPOL; ++c) {
                    float2 kr[NPOL];
                    smem_krow<NPOL, CONV ? AW_STORAGE_FP32 : ST>(sl, tl, c, kr);
#pragma unroll
                    for (int j = 0; j < VB; ++j) {
                        float re = acc[(j * NPOL + c) * 2], im = acc[(j * NPOL + c) * 2 + 1];
#pragma unroll
                        for (int s2 = 0; s2 < NPOL; ++s2) {
                            re = fmaf(kr[s2].x, gv[j][s2].x, re);
                            re = fmaf(-kr[s2].y, gv[j][s2].y, re);
                            im = fmaf(kr[s2].x, gv[j][s2].y, im);
                            im = fmaf(kr[s2].y, gv[j][s2].x, im);
                        }
                        acc[(j * NPOL + c) * 2] = re;
                        acc[(j * NPOL + c) * 2 + 1] = im;
                    }
                }
            }
            if (slab == nsl - 1) {
                // warp reduction; value index i = (j * NPOL + c) * 2 + re/im
                if constexpr (NV == 32) {
                    reduce_scatter_step<16>(acc, lane);
                    const int j = lane / (NPOL * 2), v = g + ngp * j;
                    if (v < count && AW_BOK(v < AW_DG_CHUNK, BC_D_OUT))
                        atomicAdd(&s_out[v * NPOL * 2 + (lane % (NPOL * 2))], acc[0]);
                } else {
#pragma unroll
                    for (int i = 0; i < NV; ++i)
                        for (int o = 16; o; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
                    if (lane == 0) {
#pragma unroll
                        for (int i = 0; i < NV; ++i) {
                            const int j = i / (NPOL * 2), v = g + ngp * j;
                            if (v < count && AW_BOK(v < AW_DG_CHUNK, BC_D_OUT))
                                atomicAdd(&s_out[v * NPOL * 2 + (i % (NPOL * 2))], acc[i]);
                        }
                    }
                }
                __syncthreads();
                for (int v = threadIdx.x; v < count; v += blockDim.x) {
                    if (!AW_BOK(v < AW_DG_CHUNK && start + v < a.nvalid, BC_D_REC)) continue;
                    const aw_rec r = a.rec_dg[start + v];
                    if (!AW_BOK(r.orig < a.nvis, BC_D_REC)) continue;
                    float2 out[NPOL];
#pragma unroll
                    for (int c = 0; c < NPOL; ++c)
                        out[c] = make_float2(s_out[(v * NPOL + c) * 2] * a.inv_scale,
                                             s_out[(v * NPOL + c) * 2 + 1] * a.inv_scale);
                    if (r.flip) {
#pragma unroll
                        for (int c = 0; c < NPOL; ++c) out[c].y = -out[c].y;
                        if (NPOL == 4) { float2 t = out[1]; out[1] = out[2]; out[2] = t; }
                    }
                    if constexpr (SUB) {
#pragma unroll
                        for (int c = 0; c < NPOL; ++c) {
                            const float2 o = a.sub_from[(int64_t)r.orig * NPOL + c];
                            out[c] = make_float2(o.x - out[c].x, o.y - out[c].y);
                        }
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
            __syncthreads();  // buffer `buf` and s_out are free again
            if (!has_next) break;
            if (to_next) {
                item += gridDim.x;
                cur = nxt;
                slab = 0;
                nsl = nslabs(cur);
                nxt_ok = item + gridDim.x < a.nitems;
                if (nxt_ok) nxt = load_hdr(item + gridDim.x);
            } else {
                ++slab;
            }
            buf ^= 1;
        }
    }
    // visibilities that were not gridded (outside or flagged) predict zero
    for (int64_t i = a.nvalid + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.nvis;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)a.rec[i].orig * NPOL;
#pragma unroll
        for (int c = 0; c < NPOL; ++c) a.vis_out[o + c] = SUB ? a.sub_from[o + c] : make_float2(0.f, 0.f);
    }
}

template <int NPOL, int ST>
size_t degrid_smem_bytes() {
    constexpr bool conv = NPOL == 4 && ST != AW_STORAGE_FP32;
    return 2 * (size_t)TabChunks<NPOL * NPOL, ST>::SLAB_BYTES +
           (conv ? (size_t)TabChunks<NPOL * NPOL, AW_STORAGE_FP32>::SLAB_BYTES : 0) +
           sizeof(float) * AW_DG_CHUNK * NPOL * 2;
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

template <int NPOL, int ST, bool SUB>
int launch_degrid_ts(const DegridArgs &a, int sm_count, cudaStream_t s) {
    const size_t smem = degrid_smem_bytes<NPOL, ST>();
    AW_CUDA_TRY(cudaFuncSetAttribute(degrid_items_kernel<NPOL, ST, SUB>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    AW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, degrid_items_kernel<NPOL, ST, SUB>, 256, smem));
    int64_t blocks = a.nitems;
    const int64_t cap = (int64_t)sm_count * std::max(per_sm, 1);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    degrid_items_kernel<NPOL, ST, SUB><<<(unsigned)blocks, 256, smem, s>>>(a);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

template <int NPOL, int ST>
int launch_degrid_t(const DegridArgs &a, int sm_count, cudaStream_t s) {
    return a.sub_from ? launch_degrid_ts<NPOL, ST, true>(a, sm_count, s) : launch_degrid_ts<NPOL, ST, false>(a, sm_count, s);
}


// CTAs per SM of the offset kernel that fit beside `tiles_per_sm` resident
// CTAs of the persistent tile kernel (registers, shared memory, threads), so
// that the two parts of the hybrid schedule run together in any launch order.
template <int NPOL, int ST>
int offsets_beside_tiles(int tiles_per_sm, int chunk, int alone) {
    cudaFuncAttributes ft{}, fo{};
    if (cudaFuncGetAttributes(&ft, grid_persistent_kernel<NPOL, ST>) != cudaSuccess ||
        cudaFuncGetAttributes(&fo, grid_offset_kernel<NPOL, ST>) != cudaSuccess)
        return 1;
    int dev = 0, regs_sm = 65536, smem_sm = 233472, thr_sm = 2048;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    auto regs_cta = [](int r) { return ((r + 7) / 8) * 8 * 256; };  // 256 threads, 8-register steps
    const int reserve = 1024;                                       // per-CTA shared memory the system keeps
    const int smem_t = (int)SmemLayout<NPOL>::bytes(chunk) + (int)ft.sharedSizeBytes + reserve;
    const int smem_o = (int)fo.sharedSizeBytes + reserve;
    int n = (regs_sm - tiles_per_sm * regs_cta(ft.numRegs)) / regs_cta(fo.numRegs);
    n = std::min(n, (smem_sm - tiles_per_sm * smem_t) / smem_o);
    n = std::min(n, (thr_sm - tiles_per_sm * 256) / 256);
    return std::max(1, std::min(n, alone));
}

template <int NPOL, int ST>
int launch_grid_offset_t(const GridOffArgs &a, int sm_count, cudaStream_t s, int beside_tiles = 0, int chunk = 0,
                         int fixed_ctas = 0) {
    // one wave of resident CTAs striding over the items in order, so that the
    // items in flight share bins and super-tiles (L2 locality)
    int per_sm = 1;
    AW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_offset_kernel<NPOL, ST>, 256, 0));
    if (beside_tiles > 0) per_sm = offsets_beside_tiles<NPOL, ST>(beside_tiles, chunk, std::max(per_sm, 1));
    int64_t blocks = a.nitems;
    const int64_t cap = fixed_ctas > 0 ? (int64_t)fixed_ctas : (int64_t)sm_count * std::max(per_sm, 1);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    grid_offset_kernel<NPOL, ST><<<(unsigned)blocks, 256, 0, s>>>(a);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

int launch_grid_offsets(const aw_grid_launch &L) {
    const aw_plan *p = L.plan;
    const aw_kernel_set *k = L.kset;
    GridOffArgs a;
    a.rec_dg = p->d_rec_dg;
    a.items = L.mode >= 0 ? L.items : p->d_items_dg;
    a.nitems = L.mode >= 0 ? L.nitems : p->nitems_dg;
    if (a.nitems == 0) return AW_OK;
    a.ktab = k->d_table;
    a.bin_offset = k->d_bin_offset;
    a.bin_support = k->d_bin_support;
    a.vis = reinterpret_cast<const float2 *>(L.vis);
    a.weight = L.weight;
    a.grid = reinterpret_cast<float2 *>(L.grid);
    a.N = p->N;
    a.OS = p->OS;
    a.wsum = p->d_wsum;
    a.nonfinite = p->d_nonfinite;
    a.inv_scale = 1.0f / k->scale;
    a.nvis = p->nvis;
    a.nvalid = p->nvalid;
    a.tab_elems = k->total_elems;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int st = k->spec.storage;
    // as a part of the hybrid schedule: leave room for the tile kernel's CTAs;
    // as a part of the region schedule: the CTA count the caller gives (L.ctas)
    const int bt = (L.mode >= 0 && p->tune.grid_mode == AW_GRID_HYBRID) ? p->tune.ctas_per_sm : 0;
    const int fx = (L.mode >= 0 && p->tune.grid_mode == AW_GRID_REGION) ? L.ctas : 0;
    const int ch = p->tune.chunk;
    if (p->npol == 1) {
        if (st == AW_STORAGE_FP32) return launch_grid_offset_t<1, AW_STORAGE_FP32>(a, sms, L.stream, bt, ch, fx);
        if (st == AW_STORAGE_BF16) return launch_grid_offset_t<1, AW_STORAGE_BF16>(a, sms, L.stream, bt, ch, fx);
        return launch_grid_offset_t<1, AW_STORAGE_FP16>(a, sms, L.stream, bt, ch, fx);
    }
    if (st == AW_STORAGE_FP32) return launch_grid_offset_t<4, AW_STORAGE_FP32>(a, sms, L.stream, bt, ch, fx);
    if (st == AW_STORAGE_BF16) return launch_grid_offset_t<4, AW_STORAGE_BF16>(a, sms, L.stream, bt, ch, fx);
    return launch_grid_offset_t<4, AW_STORAGE_FP16>(a, sms, L.stream, bt, ch, fx);
}

}  // namespace

int aw_launch_grid(const aw_grid_launch &L) {
    const aw_plan *p = L.plan;
    const aw_kernel_set *k = L.kset;
    if (p->nitems == 0) return AW_OK;
    const int mode = L.mode >= 0 ? L.mode : p->tune.grid_mode;
    if (mode == AW_GRID_HYBRID || mode == AW_GRID_REGION)
        return aw_set_error(AW_EINVAL, "hybrid / region schedule launched as one part");
    if (mode == AW_GRID_OFFSETS) return launch_grid_offsets(L);
    GridArgs a;
    a.rec = p->d_rec;
    a.items = L.mode >= 0 ? L.items : p->d_items;
    a.nitems = L.mode >= 0 ? L.nitems : p->nitems;
    if (a.nitems == 0) return AW_OK;
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
    a.nvis = p->nvis;
    a.nvalid = p->nvalid;
    a.tab_elems = k->total_elems;
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
                     cudaStream_t s, const void *sub_from) {
    if (p->nvis == 0) return AW_OK;
    DegridArgs a;
    a.sub_from = reinterpret_cast<const float2 *>(sub_from);
    a.rec = p->d_rec;
    a.rec_dg = p->d_rec_dg;
    a.items = p->d_items_dg;
    a.nitems = p->nitems_dg;
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
    a.tab_elems = k->total_elems;
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

// Bounds-check status of the kernels in this file: AW_EUNSUPPORTED unless the
// library was built with -DAW_BOUNDS_CHECK.
extern "C" int aw_debug_bounds_status(uint32_t *status, int32_t reset) {
    if (!status) return aw_set_error(AW_EINVAL, "status is NULL");
#ifdef AW_BOUNDS_CHECK
    unsigned int v = 0, vr = 0;
    AW_CUDA_TRY(cudaDeviceSynchronize());
    AW_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_bounds_status, sizeof(v)));
    if (reset) {
        const unsigned int z = 0;
        AW_CUDA_TRY(cudaMemcpyToSymbol(g_bounds_status, &z, sizeof(z)));
    }
    int rc = aw_region_bounds_status(&vr, reset);
    if (rc) return rc;
    *status = v ? v : vr;
    return AW_OK;
#else
    (void)reset;
    *status = 0;
    return aw_set_error(AW_EUNSUPPORTED, "built without AW_BOUNDS_CHECK");
#endif
}
