// Gridding with the learned surrogate evaluated inline: every (visibility,
// tap) point runs the SIREN MLP on tensor cores (mma.sync m16n8k16, FP16
// weights and activations, FP32 accumulation) to produce the P complex
// Mueller kernel values of that tap, which are applied to the visibility and
// added to the grid.  The kernel coordinates are continuous: the exact
// visibility position (no oversampling grid), its exact w (no w-plane
// quantisation) and the centre of its beam-frequency bin; no kernel table is read.  Items
// whose w plane the surrogate was rejected on read the exact tables instead
// (the same accumulation code, fed from memory).
//
// Sec. 3.2 of arXiv:2206.15117: the gridding kernels are the uv transforms of
// the inverse Mueller cells; here a network trained on those transforms
// supplies them.
#include <algorithm>
#include <cmath>

#include "aw_internal.h"
#include "aw_mlp.h"

namespace {

constexpr int LW = 128;        // hidden width
constexpr int LPAD = LW + 8;   // shared-memory row stride in halves (bank-conflict free ldmatrix)
constexpr int LWARPS = 8;
constexpr int LCHUNK = 128;    // staged visibilities per pass over an item

struct __align__(16) VisL {
    float2 v[4];     // flipped, weighted values
    float dx, dy;    // exact position minus footprint start, cells
    float w, f;      // |w| (wavelengths) and frequency (Hz)
    int pos;         // x0 | y0 << 16
    int koff;        // fallback table block offset (fy * OS + fx) * L * P
    float inv_off;   // 1 / offset scale for this |w|
    int pad1;
};

struct LearnArgs {
    const aw_rec *rec;
    const int4 *items;
    int64_t nitems;
    const float2 *vis;
    const float *weight;
    float2 *grid;
    int N, OS;
    // coordinates for the exact positions
    const double *uvw;
    const uint32_t *row;
    const uint16_t *chan;
    const double *freq;
    double cells_per_lambda, half_cells;
    const int32_t *bin_support;
    int npa, nfb;
    const double *pa_centres;
    int freq_channel;         // 1: the visibility's channel frequency, 0: its bin centre
    // surrogate
    const __half *Wh;
    const float *Wf;
    int64_t woff[5], boff[5];
    float omega0, w_scale, f_c, inv_f_h, chi_c, inv_chi_h, out_scale;
    double D, w_max;          // offset scale D (S(w)/2 + 1), S from the normalisation planes
    const int32_t *norm;
    int norm_nw;
    const uint8_t *plane_rejected;
    // exact fallback tables
    const void *ktab;
    const int64_t *bin_offset;
    int storage, ce;
    float inv_kscale;
    // degridding: the model grid read and the visibilities written
    const float2 *model;
    float2 *vis_out;
    int64_t nvis, nvalid;
    // statistics / queue
    double *wsum;
    unsigned long long *nonfinite;
    unsigned int *counter;
};

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float2 read_tab(const void *tab, int storage, int64_t idx) {
    if (storage == AW_STORAGE_FP32) return reinterpret_cast<const float2 *>(tab)[idx];
    if (storage == AW_STORAGE_BF16) return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(tab)[idx]);
    return __half22float2(reinterpret_cast<const __half2 *>(tab)[idx]);
}

// One 128 -> NT*8 layer for the warp's 16 rows: out = act(A W^T + b).
template <int NT>
__device__ __forceinline__ void warp_layer(const __half *sAin, const __half *sWl, const float *bias, float (&acc)[NT][4],
                                           int lane) {
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < LW / 16; ++ks) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(a0, a1, a2, a3, sAin + (lane % 16) * LPAD + ks * 16 + (lane / 16) * 8);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            uint32_t b0, b1;
            ldsm_x2(b0, b1, sWl + (nt * 8 + (lane % 8)) * LPAD + ks * 16 + ((lane / 8) % 2) * 8);
            mma16816(acc[nt], a0, a1, a2, a3, b0, b1);
        }
    }
    const int tig = lane % 4;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const float b0 = bias[nt * 8 + tig * 2], b1 = bias[nt * 8 + tig * 2 + 1];
        acc[nt][0] += b0;
        acc[nt][1] += b1;
        acc[nt][2] += b0;
        acc[nt][3] += b1;
    }
}

// Stage the visibilities [c0, c0 + cnt) of item `it` (bin `bin`, L taps):
// exact coordinates (FP64), flipped and weighted values; the weight sum and
// the non-finite count are reduced over the block and added to the plan's
// statistics.  All threads of the block call it.
template <int NPOL, bool DEG = false>
__device__ void stage_chunk(const LearnArgs &a, int4 it, int c0, int cnt, int L, int bin, VisL *sv, double *s_red) {
    constexpr int P = NPOL * NPOL;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double wloc = 0.0;
    unsigned long long nbad = 0;
    for (int i = tid; i < cnt; i += blockDim.x) {
        const aw_rec r = a.rec[it.x + c0 + i];
        const uint32_t row = a.row[r.orig];
        const uint16_t ch = a.chan[r.orig];
        const double fq = a.freq[ch];
        const double fl = fq / AW_C_LIGHT;
        double u = a.uvw[3 * (int64_t)row] * fl, v = a.uvw[3 * (int64_t)row + 1] * fl;
        double w = a.uvw[3 * (int64_t)row + 2] * fl;
        if (w < 0) { u = -u; v = -v; w = -w; }
        VisL e;
        e.dx = (float)(u * a.cells_per_lambda + a.half_cells - (double)r.x0);
        e.dy = (float)(v * a.cells_per_lambda + a.half_cells - (double)r.y0);
        e.w = (float)w;
        {
            int pn = a.w_max > 0 ? (int)floor(w * a.norm_nw / a.w_max) : 0;
            pn = min(max(pn, 0), a.norm_nw - 1);
            e.inv_off = (float)(1.0 / (a.D * (a.norm[pn] / 2 + 1)));
        }
        e.pad1 = 0;
        // the beam frequency: by default the centre of the visibility's bin
        // (the exact path averages the beam over the same channel range),
        // or the visibility's own channel frequency
        e.f = a.freq_channel ? (float)fq : (float)a.pa_centres[a.npa + bin % a.nfb];
        e.pos = (int)r.x0 | ((int)r.y0 << 16);
        e.koff = ((int)r.fy * a.OS + (int)r.fx) * L * P;
        if constexpr (DEG) {
            // degridding stages coordinates only
            for (int c = 0; c < 4; ++c) e.v[c] = make_float2(0.f, 0.f);
            sv[i] = e;
            continue;
        }
        float2 vv[4] = {};
        float ww[4] = {0, 0, 0, 0};
        bool bad = false;
        for (int c = 0; c < NPOL; ++c) {
            vv[c] = a.vis[(int64_t)r.orig * NPOL + c];
            ww[c] = a.weight ? a.weight[(int64_t)r.orig * NPOL + c] : 1.f;
            bad |= !isfinite(vv[c].x) || !isfinite(vv[c].y) || !isfinite(ww[c]);
        }
        if (r.flip) {
            for (int c = 0; c < NPOL; ++c) vv[c].y = -vv[c].y;
            if (NPOL == 4) {
                float2 t = vv[1]; vv[1] = vv[2]; vv[2] = t;
                float tw = ww[1]; ww[1] = ww[2]; ww[2] = tw;
            }
        }
        if (bad) {
            nbad++;
            for (int c = 0; c < NPOL; ++c) { vv[c] = make_float2(0.f, 0.f); ww[c] = 0.f; }
        }
        double wm = 0;
        for (int c = 0; c < 4; ++c) {
            e.v[c] = (c < NPOL) ? make_float2(ww[c] * vv[c].x, ww[c] * vv[c].y) : make_float2(0.f, 0.f);
            if (c < NPOL) wm += ww[c];
        }
        wloc += wm / NPOL;
        sv[i] = e;
    }
    if constexpr (DEG) return;   // no statistics (every thread returns here)
    for (int o = 16; o; o >>= 1) {
        wloc += __shfl_xor_sync(0xffffffffu, wloc, o);
        nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    }
    if (lane == 0) {
        s_red[warp] = wloc;
        if (nbad) atomicAdd(a.nonfinite, nbad);
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
        atomicAdd(a.wsum, t);
    }
}

template <int NPOL>
__global__ void __launch_bounds__(256, 1) grid_learned_kernel(LearnArgs a) {
    constexpr int P = NPOL * NPOL;
    constexpr int NOUT = (2 * P + 7) / 8 * 8;   // 32 (full pol) or 8 (Stokes I)
    constexpr int NTO = NOUT / 8;
    extern __shared__ __align__(16) unsigned char smem[];
    __half *sW = reinterpret_cast<__half *>(smem);             // [3][LW][LPAD]
    __half *sWo = sW + 3 * LW * LPAD;                           // [NOUT][LPAD]
    __half *sAct = sWo + NOUT * LPAD;                           // [LWARPS][2][16][LPAD]
    float *sW1 = reinterpret_cast<float *>(sAct + LWARPS * 2 * 16 * LPAD);  // [LW][5]
    float *sB = sW1 + LW * 5;                                   // [4][LW] hidden biases, then [NOUT]
    VisL *sv = reinterpret_cast<VisL *>(sB + 4 * LW + NOUT);    // [LCHUNK]
    __shared__ int s_item;
    __shared__ double s_red[LWARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- weights into shared memory once
    for (int l = 0; l < 3; ++l)
        for (int i = tid; i < LW * LW; i += blockDim.x) {
            const int o = i / LW, k = i % LW;
            sW[(l * LW + o) * LPAD + k] = a.Wh[a.woff[l + 1] + i];
        }
    for (int i = tid; i < NOUT * LW; i += blockDim.x) {
        const int o = i / LW, k = i % LW;
        sWo[o * LPAD + k] = (o < 2 * P) ? a.Wh[a.woff[4] + (int64_t)o * LW + k] : __float2half(0.f);
    }
    for (int i = tid; i < LW * 5; i += blockDim.x) sW1[i] = a.Wf[a.woff[0] + i];
    for (int i = tid; i < 4 * LW; i += blockDim.x) sB[i] = a.Wf[a.boff[i / LW] + (i % LW)];
    for (int i = tid; i < NOUT; i += blockDim.x) sB[4 * LW + i] = (i < 2 * P) ? a.Wf[a.boff[4] + i] : 0.f;
    __syncthreads();

    __half *myA = sAct + (warp * 2 + 0) * 16 * LPAD;
    __half *myB = sAct + (warp * 2 + 1) * 16 * LPAD;
    const int gid = lane >> 2, tig = lane & 3;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= a.nitems) break;
        const int4 it = a.items[item];
        const int bin = it.z;
        const int S = a.bin_support[bin];
        const int L = S * S;
        const int plane = bin / (a.npa * a.nfb);
        const int pab = (bin / a.nfb) % a.npa;
        const bool rejected = a.plane_rejected && a.plane_rejected[plane];
        const float chi_feat = (float)((a.pa_centres[pab] - a.chi_c) * a.inv_chi_h);
        const int64_t tab0 = a.bin_offset ? a.bin_offset[bin] : 0;
        for (int c0 = 0; c0 < it.y; c0 += LCHUNK) {
            const int cnt = min(LCHUNK, it.y - c0);
            __syncthreads();
            stage_chunk<NPOL>(a, it, c0, cnt, L, bin, sv, s_red);
            // ---- points of this chunk, 16 rows per warp-tile
            const int npts = cnt * L;
            for (int t0 = warp * 16; t0 < npts; t0 += LWARPS * 16) {
                // the two rows this lane owns in the fragment layout
                int vi[2], gx[2], gy[2], tap[2];
                bool ok[2];
                for (int h = 0; h < 2; ++h) {
                    const int p = t0 + gid + 8 * h;
                    ok[h] = p < npts;
                    const int pp = ok[h] ? p : 0;
                    vi[h] = pp / L;
                    tap[h] = pp - vi[h] * L;
                    const int jy = tap[h] / S, jx = tap[h] - (tap[h] / S) * S;
                    const int pos = sv[vi[h]].pos;
                    gx[h] = (pos & 0xffff) + jx;
                    gy[h] = (pos >> 16) + jy;
                }
                // K_{s, c = tig} for s = 0..NTO-1 (full pol) / K at tig == 0 (Stokes I), two rows
                float kre[2][NTO], kim[2][NTO];
                if (!rejected) {
                    // layer 1 (5 -> 128) in FP32: lane pair per row, 64 outputs each
                    {
                        const int r = lane >> 1, half = lane & 1;
                        const int p = t0 + r;
                        float x[5] = {0, 0, 0, 0, 0};
                        if (p < npts) {
                            const int i = p / L, tp = p - (p / L) * L;
                            const int jy = tp / S, jx = tp - (tp / S) * S;
                            x[0] = ((float)jx - sv[i].dx) * sv[i].inv_off;
                            x[1] = ((float)jy - sv[i].dy) * sv[i].inv_off;
                            x[2] = sv[i].w * a.w_scale - 1.f;
                            x[3] = (sv[i].f - a.f_c) * a.inv_f_h;
                            x[4] = chi_feat;
                        }
                        for (int o = half * 64; o < half * 64 + 64; o += 2) {
                            float z0 = sB[o], z1 = sB[o + 1];
#pragma unroll
                            for (int k = 0; k < 5; ++k) {
                                z0 = fmaf(sW1[o * 5 + k], x[k], z0);
                                z1 = fmaf(sW1[(o + 1) * 5 + k], x[k], z1);
                            }
                            *reinterpret_cast<__half2 *>(myA + r * LPAD + o) =
                                __floats2half2_rn(__sinf(a.omega0 * z0), __sinf(a.omega0 * z1));
                        }
                    }
                    __syncwarp();
                    // layers 2..4 on tensor cores
                    __half *src = myA, *dst = myB;
                    for (int l = 0; l < 3; ++l) {
                        float acc[LW / 8][4];
                        warp_layer<LW / 8>(src, sW + l * LW * LPAD, sB + (l + 1) * LW, acc, lane);
#pragma unroll
                        for (int nt = 0; nt < LW / 8; ++nt) {
                            const int col = nt * 8 + tig * 2;
                            *reinterpret_cast<__half2 *>(dst + gid * LPAD + col) =
                                __floats2half2_rn(__sinf(a.omega0 * acc[nt][0]), __sinf(a.omega0 * acc[nt][1]));
                            *reinterpret_cast<__half2 *>(dst + (gid + 8) * LPAD + col) =
                                __floats2half2_rn(__sinf(a.omega0 * acc[nt][2]), __sinf(a.omega0 * acc[nt][3]));
                        }
                        __syncwarp();
                        __half *t = src; src = dst; dst = t;
                    }
                    // output layer
                    float acc[NTO][4];
                    warp_layer<NTO>(src, sWo, sB + 4 * LW, acc, lane);
#pragma unroll
                    for (int nt = 0; nt < NTO; ++nt) {
                        kre[0][nt] = acc[nt][0] * a.out_scale;
                        kim[0][nt] = acc[nt][1] * a.out_scale;
                        kre[1][nt] = acc[nt][2] * a.out_scale;
                        kim[1][nt] = acc[nt][3] * a.out_scale;
                    }
                } else {
                    // fallback: the exact table values at the quantised offset
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int nt = 0; nt < NTO; ++nt) {
                            kre[h][nt] = 0.f;
                            kim[h][nt] = 0.f;
                            const int m = (NPOL == 4) ? nt * 4 + tig : 0;
                            if (ok[h] && (NPOL == 4 || tig == 0)) {
                                const float2 k = read_tab(a.ktab, a.storage,
                                                          tab0 + sv[vi[h]].koff + aw_tab_index(a.ce, L, tap[h], m));
                                kre[h][nt] = k.x * a.inv_kscale;
                                kim[h][nt] = k.y * a.inv_kscale;
                            }
                        }
                }
                // apply to the visibility and add to the grid
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 vq = sv[vi[h]].v[NPOL == 4 ? tig : 0];
                    float2 cs[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const float kr = (s < NTO) ? kre[h][s] : 0.f, ki = (s < NTO) ? kim[h][s] : 0.f;
                        cs[s] = make_float2(kr * vq.x - ki * vq.y, kr * vq.y + ki * vq.x);
                    }
                    if (NPOL == 4) {
                        // sum over the correlation c = tig held by the 4 lanes of the quad
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            cs[s].x += __shfl_xor_sync(0xffffffffu, cs[s].x, 1);
                            cs[s].y += __shfl_xor_sync(0xffffffffu, cs[s].y, 1);
                            cs[s].x += __shfl_xor_sync(0xffffffffu, cs[s].x, 2);
                            cs[s].y += __shfl_xor_sync(0xffffffffu, cs[s].y, 2);
                        }
                        if (ok[h])
                            atomicAdd(a.grid + ((int64_t)tig * a.N + gy[h]) * a.N + gx[h], cs[tig]);
                    } else if (ok[h] && tig == 0) {
                        atomicAdd(a.grid + (int64_t)gy[h] * a.N + gx[h], cs[0]);
                    }
                }
            }
        }
    }
}

// ============================================================================
// The same gridding with the network on the 5th-generation tensor cores.
//
// A CTA pushes tiles of 128 (visibility, tap) rows through the network: the
// FP16 activations of a tile (A) and the FP16 weights of every layer (B) sit
// in shared memory in the canonical K-major layout without swizzle (8 x 8
// core matrices of 128 contiguous bytes; 128 B to the next core matrix along
// K, 2048 B to the next group of 8 rows), one thread issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, K = 16 per instruction) with
// the FP32 accumulator in tensor memory, tcgen05.commit signals an mbarrier,
// and the 8 warps read the accumulator back with tcgen05.ld (warp w reaches
// TMEM lanes 32 (w % 4) ..), add the bias, take the sine and store the next
// layer's FP16 operand.  After the output layer each row's thread holds the
// P complex Mueller values of its tap and adds the product with the
// visibility to the grid.  Every mbarrier wait is bounded: a wait that runs
// out sets the error word, and the CTA leaves its loops, frees its tensor
// memory and returns.
namespace tc {

constexpr int TM = 128;                      // rows per tile (MMA M)
constexpr int KCM = LW / 8;                  // core matrices along K (16)
constexpr int TILE_BYTES = TM * LW * 2;      // 32 KB: a 128 x 128 FP16 operand
constexpr uint32_t TMEM_COLS = 512;          // 128 columns per warpgroup (at most 4)
constexpr long long WAIT_LIMIT = 1ll << 22;  // mbarrier polls (with back-off) before giving up

// byte offset of element (row r, k) of a K-major core-matrix operand with LW columns
__device__ __forceinline__ uint32_t cm_off(int r, int k) {
    return (uint32_t)(((r >> 3) * KCM + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30),
// SBO >> 4 [32,46), version 1 [46,48), no swizzle [61,64)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(2048u >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor, kind::f16: D F32 [4,6) = 1, A = B = F16 (0), both
// K-major, N >> 3 at [17,23), M >> 4 at [24,29)
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with parity `parity`; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        if (mbar_try(mbar, parity)) return true;
        if (i > 64) __nanosleep(128);
    }
    return false;
}

// 8 FP16 values of row r, columns [k0, k0 + 8), into the operand tile
__device__ __forceinline__ void st8(unsigned char *tile, int r, int k0, const float (&x)[8]) {
    uint4 q;
    __half2 h0 = __floats2half2_rn(x[0], x[1]), h1 = __floats2half2_rn(x[2], x[3]);
    __half2 h2 = __floats2half2_rn(x[4], x[5]), h3 = __floats2half2_rn(x[6], x[7]);
    q.x = *reinterpret_cast<uint32_t *>(&h0);
    q.y = *reinterpret_cast<uint32_t *>(&h1);
    q.z = *reinterpret_cast<uint32_t *>(&h2);
    q.w = *reinterpret_cast<uint32_t *>(&h3);
    *reinterpret_cast<uint4 *>(tile + cm_off(r, k0)) = q;
}

}  // namespace tc

// Self-test of the bounded mbarrier wait: an mbarrier that nothing arrives on.
__global__ void mbar_timeout_kernel(unsigned int *err) {
    __shared__ __align__(8) unsigned long long mbar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::su32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(tc::su32(&mbar), 0)) atomicExch(err, 1u);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(tc::su32(&mbar)) : "memory");
}

template <int NPOL>
struct TcDims {
    static constexpr int P = NPOL * NPOL;
    static constexpr int NOUT = (2 * P + 15) / 16 * 16;   // 32 (full pol) or 16 (Stokes I): MMA N
    static constexpr size_t W_OFF = 0;                                  // 3 hidden layers, 32 KB each
    static constexpr size_t WO_OFF = 3 * (size_t)tc::TILE_BYTES;        // output layer [NOUT][LW]
    static constexpr int NWG = 3;                                       // warpgroups (tiles in flight)
    static constexpr size_t A_OFF = WO_OFF + (size_t)NOUT * LW * 2;     // one activation tile per warpgroup
    static constexpr size_t W1_OFF = A_OFF + NWG * (size_t)tc::TILE_BYTES;  // float [LW][5]
    static constexpr size_t B_OFF = W1_OFF + (size_t)LW * 5 * 4;        // float [4][LW] omega0 x bias, then [NOUT] bias
    static constexpr size_t SV_OFF = (B_OFF + (size_t)(4 * LW + NOUT) * 4 + 15) / 16 * 16;
    static constexpr size_t BYTES = SV_OFF + (size_t)LCHUNK * sizeof(VisL);
};

__device__ __forceinline__ void wg_sync(int wg) {
    asm volatile("bar.sync %0, 128;\n" ::"r"(1 + wg) : "memory");
}

// The NWG warpgroups of the CTA work on interleaved tiles of a chunk, each
// with its own activation tile, 128 accumulator columns (the output layer
// reuses the first 32 once the last hidden epilogue has read them) and
// mbarrier, and an elected thread of each issues its own MMAs: while some
// warpgroups run epilogues the tensor cores work on another's layer.
//
// DEG: degridding with the same network evaluation.  A point (visibility,
// tap) gathers the npol model values at its cell and forms sum_s K_{c,s} G_s;
// the lanes of a warp that hold the same visibility (contiguous) are summed by
// a segmented shuffle scan and the segment heads add into the chunk's
// shared-memory accumulators; the chunk's visibilities are then written out
// (un-flipped), and the visibilities outside the plan's valid range get 0.
template <int NPOL, bool DEG>
__global__ void __launch_bounds__(128 * TcDims<NPOL>::NWG, 1) grid_learned_tc_kernel(LearnArgs a, unsigned int *err) {
    using Dm = TcDims<NPOL>;
    constexpr int NWG = Dm::NWG;
    constexpr int P = Dm::P;
    constexpr int NOUT = Dm::NOUT;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *sW = smem + Dm::W_OFF;
    unsigned char *sWo = smem + Dm::WO_OFF;
    float *sW1 = reinterpret_cast<float *>(smem + Dm::W1_OFF);
    float *sB = reinterpret_cast<float *>(smem + Dm::B_OFF);
    VisL *sv = reinterpret_cast<VisL *>(smem + Dm::SV_OFF);
    __shared__ __align__(8) unsigned long long s_mbar[NWG];
    __shared__ uint32_t s_tmem;
    __shared__ int s_item, s_abort, s_wgab[NWG];
    __shared__ double s_red[4 * NWG];
    __shared__ float2 s_acc[DEG ? LCHUNK * NPOL : 1];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int wg = warp >> 2, wtid = tid & 127;          // warpgroup, thread within it (= tile row)
    unsigned char *sA = smem + Dm::A_OFF + (size_t)wg * tc::TILE_BYTES;

    // ---- weights into the operand layouts once
    for (int l = 0; l < 3; ++l)
        for (int i = tid; i < LW * LW; i += blockDim.x) {
            const int o = i / LW, k = i % LW;
            *reinterpret_cast<__half *>(sW + (size_t)l * tc::TILE_BYTES + tc::cm_off(o, k)) = a.Wh[a.woff[l + 1] + i];
        }
    for (int i = tid; i < NOUT * LW; i += blockDim.x) {
        const int o = i / LW, k = i % LW;
        *reinterpret_cast<__half *>(sWo + tc::cm_off(o, k)) =
            (o < 2 * P) ? a.Wh[a.woff[4] + (int64_t)o * LW + k] : __float2half(0.f);
    }
    for (int i = tid; i < LW * 5; i += blockDim.x) sW1[i] = a.Wf[a.woff[0] + i];
    for (int i = tid; i < 4 * LW; i += blockDim.x) {
        const float b = a.Wf[a.boff[i / LW] + (i % LW)];
        sB[i] = (i < LW) ? b : a.omega0 * b;   // layer 1 keeps the plain bias (FP32 layer)
    }
    for (int i = tid; i < NOUT; i += blockDim.x) sB[4 * LW + i] = (i < 2 * P) ? a.Wf[a.boff[4] + i] : 0.f;
    if (tid == 0) {
        for (int g = 0; g < NWG; ++g) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::su32(&s_mbar[g])) : "memory");
            s_wgab[g] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::su32(&s_tmem)),
                     "r"(tc::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t acc_h = tmem + (uint32_t)wg * 128;        // this warpgroup's accumulator columns
    const uint32_t acc_o = acc_h;                            // the output layer (N <= 32) reuses them
    const uint32_t id_h = tc::idesc(tc::TM, LW), id_o = tc::idesc(tc::TM, NOUT);
    const uint32_t aA = tc::su32(sA), aW = tc::su32(sW), aWo = tc::su32(sWo);
    const uint32_t mbar = tc::su32(&s_mbar[wg]);
    uint32_t phase = 0;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= a.nitems || s_abort) break;
        const int4 it = a.items[item];
        const int bin = it.z;
        const int S = a.bin_support[bin];
        const int L = S * S;
        const int plane = bin / (a.npa * a.nfb);
        const int pab = (bin / a.nfb) % a.npa;
        const bool rejected = a.plane_rejected && a.plane_rejected[plane];
        const float chi_feat = (float)((a.pa_centres[pab] - a.chi_c) * a.inv_chi_h);
        const int64_t tab0 = a.bin_offset ? a.bin_offset[bin] : 0;
        for (int c0 = 0; c0 < it.y && !s_abort; c0 += LCHUNK) {
            const int cnt = min(LCHUNK, it.y - c0);
            __syncthreads();
            stage_chunk<NPOL, DEG>(a, it, c0, cnt, L, bin, sv, s_red);
            if constexpr (DEG)
                for (int i = tid; i < cnt * NPOL; i += blockDim.x) s_acc[i] = make_float2(0.f, 0.f);
            __syncthreads();
            const int npts = cnt * L;
            // this warpgroup's tiles: NWG k + wg
            for (int t0 = wg * tc::TM; t0 < npts; t0 += NWG * tc::TM) {
                const int p = t0 + wtid;
                const bool okp = p < npts;
                const int vi = okp ? p / L : 0;
                const int tp = okp ? p - vi * L : 0;
                const int jy = tp / S, jx = tp - (tp / S) * S;
                float kv[2 * P];
                if (!rejected) {
                    // layer 1 (5 -> 128) in FP32, one row per thread
                    {
                        float x[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                        if (okp) {
                            x[0] = ((float)jx - sv[vi].dx) * sv[vi].inv_off;
                            x[1] = ((float)jy - sv[vi].dy) * sv[vi].inv_off;
                            x[2] = sv[vi].w * a.w_scale - 1.f;
                            x[3] = (sv[vi].f - a.f_c) * a.inv_f_h;
                            x[4] = chi_feat;
                        }
                        for (int g = 0; g < LW / 8; ++g) {
                            float h[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int o = g * 8 + e;
                                float z = sB[o];
#pragma unroll
                                for (int k = 0; k < 5; ++k) z = fmaf(sW1[o * 5 + k], x[k], z);
                                h[e] = __sinf(a.omega0 * z);
                            }
                            tc::st8(sA, wtid, g * 8, h);
                        }
                    }
                    tc::fence_smem_async();
                    tc::fence_before();
                    wg_sync(wg);
                    // layers 2..4 and the output layer
                    for (int l = 0; l < 4; ++l) {
                        const bool out_layer = (l == 3);
                        if (wtid == 0) {
                            tc::fence_after();
                            const uint32_t wb = out_layer ? aWo : aW + (uint32_t)l * tc::TILE_BYTES;
#pragma unroll
                            for (int ks = 0; ks < LW / 16; ++ks)
                                tc::mma(out_layer ? acc_o : acc_h, tc::sdesc(aA + ks * 256), tc::sdesc(wb + ks * 256),
                                        out_layer ? id_o : id_h, ks > 0 ? 1u : 0u);
                            tc::commit(mbar);
                        }
                        const bool done = tc::mbar_wait(mbar, phase);
                        phase ^= 1u;
                        if (!done) {
                            atomicExch(err, 1u);
                            s_wgab[wg] = 1;
                        }
                        tc::fence_after();
                        if (!out_layer) {
                            // this row's 128 columns: omega0 (acc + bias), sine, FP16 operand
                            const float *bw = sB + (l + 1) * LW;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                float v[32];
                                tc::ld32(acc_h + lane_base + 32 * q, v);
#pragma unroll
                                for (int g = 0; g < 4; ++g) {
                                    float h[8];
#pragma unroll
                                    for (int e = 0; e < 8; ++e) {
                                        const int c = 32 * q + g * 8 + e;
                                        h[e] = __sinf(fmaf(a.omega0, v[g * 8 + e], bw[c]));
                                    }
                                    tc::st8(sA, wtid, 32 * q + g * 8, h);
                                }
                            }
                            tc::fence_smem_async();
                        } else {
                            float v[32];
                            tc::ld32(acc_o + lane_base, v);
#pragma unroll
                            for (int i = 0; i < 2 * P; ++i) kv[i] = (v[i] + sB[4 * LW + i]) * a.out_scale;
                        }
                        tc::fence_before();
                        wg_sync(wg);
                        if (s_wgab[wg]) break;   // read after the barrier: the same in every thread
                    }
                } else {
                    // rejected plane: the exact table values at the quantised offset
#pragma unroll
                    for (int m = 0; m < P; ++m) {
                        float2 k = make_float2(0.f, 0.f);
                        if (okp) k = read_tab(a.ktab, a.storage, tab0 + sv[vi].koff + aw_tab_index(a.ce, L, tp, m));
                        kv[2 * m] = k.x * a.inv_kscale;
                        kv[2 * m + 1] = k.y * a.inv_kscale;
                    }
                }
                if (s_wgab[wg]) break;
                if constexpr (DEG) {
                    // sum_s K_{c,s} G_s at this point's cell
                    float2 o[NPOL];
#pragma unroll
                    for (int c = 0; c < NPOL; ++c) o[c] = make_float2(0.f, 0.f);
                    if (okp) {
                        const int pos = sv[vi].pos;
                        const int gx = (pos & 0xffff) + jx, gy = (pos >> 16) + jy;
                        float2 gv[NPOL];
#pragma unroll
                        for (int s2 = 0; s2 < NPOL; ++s2) gv[s2] = __ldg(a.model + ((int64_t)s2 * a.N + gy) * a.N + gx);
#pragma unroll
                        for (int c = 0; c < NPOL; ++c)
#pragma unroll
                            for (int s2 = 0; s2 < NPOL; ++s2) {
                                const float kr = kv[2 * (c * NPOL + s2)], ki = kv[2 * (c * NPOL + s2) + 1];
                                o[c].x += kr * gv[s2].x - ki * gv[s2].y;
                                o[c].y += kr * gv[s2].y + ki * gv[s2].x;
                            }
                    }
                    // segmented suffix scan over the warp: lanes holding one visibility are
                    // contiguous; lanes past the chunk get keys of their own
                    const int lane = tid & 31;
                    const int key = okp ? vi : (1 << 24) + lane;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int ko = __shfl_down_sync(0xffffffffu, key, off);
                        const bool same = lane + off < 32 && ko == key;
#pragma unroll
                        for (int c = 0; c < NPOL; ++c) {
                            const float tx = __shfl_down_sync(0xffffffffu, o[c].x, off);
                            const float ty = __shfl_down_sync(0xffffffffu, o[c].y, off);
                            if (same) { o[c].x += tx; o[c].y += ty; }
                        }
                    }
                    const int kp = __shfl_up_sync(0xffffffffu, key, 1);
                    if (okp && (lane == 0 || kp != key)) {
#pragma unroll
                        for (int c = 0; c < NPOL; ++c) {
                            atomicAdd(&s_acc[vi * NPOL + c].x, o[c].x);
                            atomicAdd(&s_acc[vi * NPOL + c].y, o[c].y);
                        }
                    }
                    continue;
                }
                // apply to the visibility and add to the grid, one row per thread
                if (okp) {
                    const int pos = sv[vi].pos;
                    const int gx = (pos & 0xffff) + jx, gy = (pos >> 16) + jy;
#pragma unroll
                    for (int so = 0; so < NPOL; ++so) {
                        float2 o = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < NPOL; ++c) {
                            const float kr = kv[2 * (so * NPOL + c)], ki = kv[2 * (so * NPOL + c) + 1];
                            const float2 vq = sv[vi].v[c];
                            o.x += kr * vq.x - ki * vq.y;
                            o.y += kr * vq.y + ki * vq.x;
                        }
                        atomicAdd(a.grid + ((int64_t)so * a.N + gy) * a.N + gx, o);
                    }
                }
            }
            __syncthreads();
            if (tid == 0)
                for (int g = 0; g < NWG; ++g)
                    if (s_wgab[g]) s_abort = 1;
            if constexpr (DEG) {
                // the chunk's visibilities, un-flipped: V -> P conj(V)
                for (int i = tid; i < cnt; i += blockDim.x) {
                    const aw_rec r = a.rec[it.x + c0 + i];
                    float2 out[NPOL];
#pragma unroll
                    for (int c = 0; c < NPOL; ++c) out[c] = s_acc[i * NPOL + c];
                    if (r.flip) {
#pragma unroll
                        for (int c = 0; c < NPOL; ++c) out[c].y = -out[c].y;
                        if (NPOL == 4) { const float2 t = out[1]; out[1] = out[2]; out[2] = t; }
                    }
#pragma unroll
                    for (int c = 0; c < NPOL; ++c) a.vis_out[(int64_t)r.orig * NPOL + c] = out[c];
                }
            }
            __syncthreads();   // s_abort is read by every thread in the loop conditions
        }
    }
    if constexpr (DEG) {
        // visibilities that were not gridded (outside or flagged) predict zero
        for (int64_t i = a.nvalid + (int64_t)blockIdx.x * blockDim.x + tid; i < a.nvis;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t o = (int64_t)a.rec[i].orig * NPOL;
#pragma unroll
            for (int c = 0; c < NPOL; ++c) a.vis_out[o + c] = make_float2(0.f, 0.f);
        }
    }
    // ---- free the tensor memory (every commit was waited for)
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tc::TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

// Run mbar_timeout_kernel: AW_ETIMEOUT once the wait has given up.
int aw_mbar_selftest(cudaStream_t st) {
    unsigned int *d = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&d, sizeof(unsigned int)));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        mbar_timeout_kernel<<<1, 32, 0, st>>>(d);
        e = cudaGetLastError();
    }
    unsigned int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    aw_dev_free(d);
    if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "mbarrier self-test: %s", cudaGetErrorString(e));
    return h ? aw_set_error(AW_ETIMEOUT, "mbarrier wait gave up") : AW_OK;
}

size_t aw_learned_smem_bytes(int npol) {
    const int P = npol * npol;
    const int NOUT = (2 * P + 7) / 8 * 8;
    return (size_t)(3 * LW * LPAD + NOUT * LPAD + LWARPS * 2 * 16 * LPAD) * sizeof(__half) +
           (size_t)(LW * 5 + 4 * LW + NOUT) * sizeof(float) + (size_t)LCHUNK * sizeof(VisL);
}

int aw_launch_grid_learned(const aw_plan *p, aw_surrogate *s, const aw_kernel_set *fallback, const uint8_t *d_rejected,
                           const double *d_pa, const void *vis, const float *weight, void *grid, const void *model,
                           void *vis_out, int sm_count, cudaStream_t st) {
    const bool deg = model != nullptr;
    if (s->cfg.width != LW || s->cfg.n_hidden != 4)
        return aw_set_error(AW_EUNSUPPORTED, "inline evaluation needs width 128 and 4 sine layers");
    if (s->cfg.npol != p->npol) return aw_set_error(AW_EINVAL, "surrogate npol %d, plan npol %d", s->cfg.npol, p->npol);
    if (deg && s->engine != AW_ENGINE_TCGEN05)
        return aw_set_error(AW_EUNSUPPORTED, "inline degridding runs on the TCGEN05 engine only");
    if (deg ? p->nvis == 0 : p->nitems == 0) return AW_OK;
    LearnArgs a;
    a.rec = p->d_rec;
    a.items = p->d_items;
    a.nitems = p->nitems;
    a.vis = reinterpret_cast<const float2 *>(vis);
    a.weight = weight;
    a.grid = reinterpret_cast<float2 *>(grid);
    a.model = reinterpret_cast<const float2 *>(model);
    a.vis_out = reinterpret_cast<float2 *>(vis_out);
    a.nvis = p->nvis;
    a.nvalid = p->nvalid;
    a.N = p->N;
    a.OS = p->OS;
    a.uvw = p->vis.uvw;
    a.row = p->vis.row_of_vis;
    a.chan = p->vis.chan_of_vis;
    a.freq = p->vis.freq;
    a.cells_per_lambda = p->uscale / p->OS;
    a.half_cells = p->N / 2;
    a.bin_support = fallback->d_bin_support;
    a.npa = fallback->spec.npa;
    a.nfb = fallback->spec.nfb;
    a.pa_centres = d_pa;
    a.freq_channel = s->freq_mode == AW_FREQ_CHANNEL;
    a.Wh = s->d_ph;
    a.Wf = s->d_p;
    for (int l = 0; l < 5; ++l) {
        a.woff[l] = s->woff[l];
        a.boff[l] = s->boff[l];
    }
    a.omega0 = s->cfg.omega0;
    a.D = s->cfg.D;
    a.norm = s->d_norm;
    a.norm_nw = (int)s->norm.size();
    a.w_max = s->cfg.w_max;
    a.w_scale = (float)(s->cfg.w_max > 0 ? 2.0 / s->cfg.w_max : 0.0);
    a.f_c = (float)s->cfg.f_c;
    a.inv_f_h = (float)(1.0 / s->cfg.f_h);
    a.chi_c = (float)s->cfg.chi_c;
    a.inv_chi_h = (float)(1.0 / s->cfg.chi_h);
    a.out_scale = s->cfg.out_scale;
    a.plane_rejected = d_rejected;
    a.ktab = fallback->d_table;
    a.bin_offset = fallback->d_bin_offset;
    a.storage = fallback->spec.storage;
    a.ce = fallback->ce;
    a.inv_kscale = 1.0f / fallback->scale;
    a.wsum = p->d_wsum;
    a.nonfinite = p->d_nonfinite;
    a.counter = p->d_counter;
    if (!deg) {
        AW_CUDA_TRY(cudaMemsetAsync(p->d_wsum, 0, sizeof(double), st));
        AW_CUDA_TRY(cudaMemsetAsync(p->d_nonfinite, 0, sizeof(unsigned long long), st));
    }
    AW_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int), st));
    const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(p->nitems, sm_count));
    if (s->engine == AW_ENGINE_TCGEN05) {
        if (!s->d_err) AW_CUDA_TRY(aw_dev_malloc(&s->d_err, sizeof(unsigned int)));
        AW_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned int), st));
        auto launch = [&](auto kern, size_t bytes, int threads) -> int {
            AW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
            kern<<<ctas, threads, bytes, st>>>(a, s->d_err);
            return AW_OK;
        };
        int lrc;
        if (p->npol == 4)
            lrc = deg ? launch(grid_learned_tc_kernel<4, true>, TcDims<4>::BYTES, 128 * TcDims<4>::NWG)
                      : launch(grid_learned_tc_kernel<4, false>, TcDims<4>::BYTES, 128 * TcDims<4>::NWG);
        else
            lrc = deg ? launch(grid_learned_tc_kernel<1, true>, TcDims<1>::BYTES, 128 * TcDims<1>::NWG)
                      : launch(grid_learned_tc_kernel<1, false>, TcDims<1>::BYTES, 128 * TcDims<1>::NWG);
        if (lrc) return lrc;
        AW_CHECK_LAUNCH();
        unsigned int e = 0;
        AW_CUDA_TRY(cudaMemcpyAsync(&e, s->d_err, sizeof(e), cudaMemcpyDeviceToHost, st));
        AW_CUDA_TRY(cudaStreamSynchronize(st));
        if (e) return aw_set_error(AW_ETIMEOUT, "%s: a tensor-core completion wait gave up; output invalid",
                                   deg ? "degrid_learned" : "grid_learned");
        return AW_OK;
    }
    const size_t smem = aw_learned_smem_bytes(p->npol);
    if (p->npol == 4) {
        AW_CUDA_TRY(cudaFuncSetAttribute(grid_learned_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grid_learned_kernel<4><<<ctas, 256, smem, st>>>(a);
    } else {
        AW_CUDA_TRY(cudaFuncSetAttribute(grid_learned_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        grid_learned_kernel<1><<<ctas, 256, smem, st>>>(a);
    }
    AW_CHECK_LAUNCH();
    return AW_OK;
}
