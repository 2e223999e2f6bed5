// Gridding, REGION schedule: one CTA accumulates a whole grid tile in shared
// memory.
//
// arXiv:2206.15117 Sec. 3.2: every visibility is convolved onto the uv grid
// with the oversampled kernel of its bin, G_s[y0 + jy][x0 + jx] +=
// sum_c K_{s,c}(jy, jx; fy, fx) w_c V_c (Sec. 2.1: w-projection planes; Sec. 3.2:
// the Mueller-cell kernels of the A term).
//
// Work item: the visibilities of one bin whose footprints start inside one
// T x T tile of the grid (at most AW_RG_MAXV of them; longer runs are cut).
// The CTA owns the tile's output region, R x R cells with R = T + S - 1, as
// FP32 accumulators in shared memory (planes (0, 1) and (2, 3) of a cell as
// two float4, so that the 8 lanes of each phase of a 128-bit access read 128
// contiguous bytes).  The items' visibilities are sorted by oversampled offset
// (fy, fx), then by the residue of their footprint row modulo M, then by
// position.
//
// Visibilities of one offset share one kernel block.  The CTA has M warps;
// warp w takes the taps whose row jy = w (mod M), S/M rows of S taps, 32 at a
// time (a "pass").  A unit is one offset group and one pass: each lane holds
// the 16 complex Mueller values of its tap in registers and, for every
// visibility of the group in turn, adds K V to the region cell the tap lands
// on with a plain shared-memory read-modify-write.  For visibilities whose
// footprint rows y0 share one residue c modulo M, warp w only ever writes
// region rows = c + w (mod M): different warps never touch the same cell, so
// the warps run through such a run of visibilities independently; the lanes of
// a warp step through the visibilities together (distinct taps, distinct
// cells).  A CTA barrier is needed only where the residue changes and at the
// end of a unit.  When the item's visibilities are done, the region is added
// to the grid in HBM (one vector atomic per plane and non-zero cell).
//
// Per visibility-tap: 64 FMAs (the products formed while the region cell is
// being read), two 16-byte shared loads and stores of the region, a broadcast
// read of the visibility; the kernel block is read from L2 once per (group,
// pass) instead of once per visibility.  Tile sizes are chosen per support so
// that the region fits two CTAs per SM (R <= AW_RG_RMAX).
#include <algorithm>

#include "aw_internal.h"

// Checked builds (-DAW_BOUNDS_CHECK): a bad index records a code here (the
// first one wins) and the access is skipped; aw_debug_bounds_status reports it.
#ifdef AW_BOUNDS_CHECK
__device__ unsigned int g_bounds_status_rg;
#endif

namespace {

#ifdef AW_BOUNDS_CHECK
__device__ __forceinline__ bool rg_bounds_ok(bool ok, unsigned int code) {
    if (!ok) atomicCAS(&g_bounds_status_rg, 0u, code);
    return ok;
}
#define RG_BOK(cond, code) rg_bounds_ok((cond), (code))
#else
#define RG_BOK(cond, code) true
#endif

enum : unsigned int { BC_R_REC = 14, BC_R_CELL, BC_R_TAB, BC_R_GRID, BC_R_SMEM };

constexpr int RG_CH = 128;      // visibilities staged per round
constexpr int RG_TPL1 = 18;     // most taps a lane in the Stokes-I form ((48 / 4) 48 / 32)
constexpr int RG_MAXT = 320;    // largest CTA (10 warps)
// resident CTAs per SM the register budget is set for (the region size,
// AW_RG_RMAX, decides the shared-memory side)
#ifndef AW_RG_MINB
#define AW_RG_MINB 2
#endif

struct RegionArgs {
    const aw_rec *rec;          // region order
    const int4 *items;          // {start, count, bin, (tile row << 16) | tile column}
    int64_t nitems;
    unsigned int *counter;      // work-queue head (zeroed before the launch)
    const void *ktab;
    const int64_t *bin_offset;
    const int32_t *bin_support;
    const float2 *vis;
    const float *weight;
    float2 *grid;
    int N, OS;
    int S, T, R;                // support, tile side and region side of this launch's items
    int M, passes;              // row classes (= warps) and passes of 32 taps per warp
    double *wsum;
    unsigned long long *nonfinite;
    float inv_scale;
    int64_t nvis, nvalid, tab_elems;
};

template <int ST>
struct RgK;
template <>
struct RgK<AW_STORAGE_FP32> {
    // 16 complex values of tap t: 8 chunks of 2, chunk c at ((c L + t) 2)
    static __device__ __forceinline__ void load(const void *base, int64_t idx, int L, int t, float2 (&k)[16]) {
        const float2 *p = reinterpret_cast<const float2 *>(base) + idx;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(p + 2 * ((int64_t)c * L + t)));
            k[2 * c] = make_float2(v.x, v.y);
            k[2 * c + 1] = make_float2(v.z, v.w);
        }
    }
};
template <int ST>
struct RgK16 {
    // 16-bit storage: 4 chunks of 4 complex values, widened to FP32 once per unit
    static __device__ __forceinline__ void load(const void *base, int64_t idx, int L, int t, float2 (&k)[16]) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(base) + idx;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + 4 * ((int64_t)c * L + t)));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if constexpr (ST == AW_STORAGE_BF16)
                    k[4 * c + j] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[j]));
                else
                    k[4 * c + j] = __half22float2(*reinterpret_cast<const __half2 *>(&w[j]));
            }
        }
    }
};
template <>
struct RgK<AW_STORAGE_BF16> : RgK16<AW_STORAGE_BF16> {};
template <>
struct RgK<AW_STORAGE_FP16> : RgK16<AW_STORAGE_FP16> {};

// Stokes I (one value per tap, one per table element): tap t at idx + t
template <int ST>
__device__ __forceinline__ float2 rg_k1(const void *base, int64_t idx, int t) {
    if constexpr (ST == AW_STORAGE_FP32) {
        return __ldg(reinterpret_cast<const float2 *>(base) + idx + t);
    } else {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(base) + idx + t);
        if constexpr (ST == AW_STORAGE_BF16) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
        else return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
}

__device__ __forceinline__ void cmac2(float &re, float &im, float2 k, float vr, float vi) {
    re = fmaf(k.x, vr, re);
    re = fmaf(-k.y, vi, re);
    im = fmaf(k.x, vi, im);
    im = fmaf(k.y, vr, im);
}

// Shared memory of one CTA: the region (R rows of NPOL complex FP32
// accumulators per cell, R cells a row plus two of padding for Stokes I), the
// staged visibilities (NPOL complex each) and four int arrays of the round.
constexpr size_t region_smem_bytes(int R, int npol) {
    return (size_t)R * (npol == 1 ? R + 2 : R) * npol * 8 + (size_t)RG_CH * npol * 8 +
           (size_t)RG_CH * 2 * sizeof(int) + (size_t)(RG_CH + 1) * 2 * sizeof(int);
}

// One full-polarisation visibility-tap on a region cell held in registers
// (planes (0, 1) in r01, (2, 3) in r23): += K V, plane s getting the sum over
// correlations c of K[s][c] V_c.
__device__ __forceinline__ void mueller_acc(float4 &r01, float4 &r23, const float2 (&k)[16], float4 v01,
                                            float4 v23) {
    cmac2(r01.x, r01.y, k[0], v01.x, v01.y);
    cmac2(r01.z, r01.w, k[4], v01.x, v01.y);
    cmac2(r23.x, r23.y, k[8], v01.x, v01.y);
    cmac2(r23.z, r23.w, k[12], v01.x, v01.y);
    cmac2(r01.x, r01.y, k[1], v01.z, v01.w);
    cmac2(r01.z, r01.w, k[5], v01.z, v01.w);
    cmac2(r23.x, r23.y, k[9], v01.z, v01.w);
    cmac2(r23.z, r23.w, k[13], v01.z, v01.w);
    cmac2(r01.x, r01.y, k[2], v23.x, v23.y);
    cmac2(r01.z, r01.w, k[6], v23.x, v23.y);
    cmac2(r23.x, r23.y, k[10], v23.x, v23.y);
    cmac2(r23.z, r23.w, k[14], v23.x, v23.y);
    cmac2(r01.x, r01.y, k[3], v23.z, v23.w);
    cmac2(r01.z, r01.w, k[7], v23.z, v23.w);
    cmac2(r23.x, r23.y, k[11], v23.z, v23.w);
    cmac2(r23.z, r23.w, k[15], v23.z, v23.w);
}

// NPOL = 4: full polarisation, 16 Mueller values a tap, units of one offset
// group and one pass of 32 taps a warp; with TMAX = 2 or 3 (CTAs of at most
// 256 or 192 threads, supports of two or three passes or more) a unit takes
// TMAX passes at once, so each visibility gives a lane TMAX independent
// read-modify-writes.  NPOL = 1: Stokes I, one value a tap
// and one plane (an eighth of the shared memory); a single update per
// visibility-tap leaves each read-modify-write little arithmetic to hide its
// latency behind, so the CTA has only 4 warps (row classes), a lane takes
// all its taps at once (a.passes of them, at most TMAX: taps lane, lane + 32,
// ... of its warp's rows) and a unit is a whole offset group: a.passes
// independent updates per visibility and lane.
template <int ST, int R, int NPOL, int TMAX>
__global__ void __launch_bounds__(NPOL == 1 ? 128 : (TMAX == 3 ? 192 : TMAX == 2 ? 256 : RG_MAXT),
                                  NPOL == 4 ? AW_RG_MINB : 4)
    grid_region_kernel(RegionArgs a) {
    // row stride of the region in cells: Stokes I pads two cells, so that region
    // rows 4 apart (the row classes of one pass of a half-warp) fall on the other
    // half of the shared-memory banks (8-byte cells, 4 rows of 58 cells = 464 words)
    constexpr int RS = NPOL == 1 ? R + 2 : R;
    constexpr int P = NPOL * NPOL, RR = R * RS;
    extern __shared__ __align__(16) char rg_smem[];
    const int S = a.S, L = S * S, M = a.M, passes = a.passes;
    // NPOL 4: planes (0, 1) and (2, 3) of a cell as two float4; NPOL 1: one float2
    float4 *reg01 = reinterpret_cast<float4 *>(rg_smem);
    float4 *reg23 = reg01 + RR;
    float2 *reg0 = reinterpret_cast<float2 *>(rg_smem);
    char *after_region = rg_smem + (size_t)RR * NPOL * 8;
    float4 *s_v = reinterpret_cast<float4 *>(after_region);     // NPOL 4: [RG_CH][2]
    float2 *s_v1 = reinterpret_cast<float2 *>(after_region);    // NPOL 1: [RG_CH]
    int *s_cell = reinterpret_cast<int *>(after_region + (size_t)RG_CH * NPOL * 8);   // [RG_CH] ly * RS + lx
    int *s_key = s_cell + RG_CH;                                // [RG_CH] offset * 64 + ly mod M
    int *s_ss = s_key + RG_CH;                                  // [RG_CH + 1] sub-group starts
    int *s_gss = s_ss + RG_CH + 1;                              // [RG_CH + 1] first sub-group of each group
    __shared__ int s_wcs[RG_CH / 32], s_wcg[RG_CH / 32];
    __shared__ int s_item, s_ng;
    __shared__ double s_red[RG_MAXT / 32];
    __shared__ unsigned long long s_redn[RG_MAXT / 32];
    const int tid = threadIdx.x, BT = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t plane = (int64_t)a.N * a.N;
    double wloc = 0.0;
    unsigned long long nbad = 0;

    for (;;) {
        __syncthreads();   // the previous item's flush is done with the region
        if (tid == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= a.nitems) break;
        const int4 it = a.items[item];
        const int start = it.x, count = it.y, bin = it.z;
        const int oy = (it.w >> 16) * a.T, ox = (it.w & 0xffff) * a.T;   // grid origin of the region
        const int64_t tab0 = a.bin_offset[bin];
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (NPOL == 4) {
            for (int c = tid; c < RR; c += BT) { reg01[c] = z4; reg23[c] = z4; }
        } else {
            for (int c = tid; c < RR; c += BT) reg0[c] = make_float2(0.f, 0.f);
        }

        // a round stages one visibility a thread: at most RG_CH, and no more
        // than the CTA's threads (the Stokes-I form runs 64-thread CTAs)
        const int round = min(RG_CH, BT), nwr = round / 32;
        for (int c0 = 0; c0 < count; c0 += round) {
            const int n = min(round, count - c0);
            __syncthreads();   // the region is zeroed / the previous round's readers are done
            // ---- stage the round's visibilities (flipped, weighted, NaN-checked)
            if (tid < n) {
                const int64_t ri = (int64_t)start + c0 + tid;
                aw_rec r{};
                if (RG_BOK(ri < a.nvalid, BC_R_REC)) r = a.rec[ri];
                const int64_t orig = RG_BOK(r.orig < a.nvis, BC_R_REC) ? (int64_t)r.orig : 0;
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
                    if constexpr (NPOL == 4) {
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
                    v[c] = make_float2(ws * v[c].x, ws * v[c].y);
                }
                wloc += wm / NPOL;
                if constexpr (NPOL == 4) {
                    s_v[2 * tid] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
                    s_v[2 * tid + 1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
                } else {
                    s_v1[tid] = v[0];
                }
                const int ly = (int)r.y0 - oy, lx = (int)r.x0 - ox;
                const bool inr = RG_BOK(ly >= 0 && lx >= 0 && ly + S <= R && lx + S <= R, BC_R_CELL);
                s_cell[tid] = inr ? ly * RS + lx : 0;
                s_key[tid] = ((int)r.fy * a.OS + (int)r.fx) * 64 + (inr ? ly % M : 0);
            }
            __syncthreads();
            // ---- offset groups (runs of equal offset) and, inside them,
            // sub-groups (runs of equal footprint-row residue)
            const bool fs = tid < n && (tid == 0 || s_key[tid] != s_key[tid - 1]);
            const bool fg = tid < n && (tid == 0 || (s_key[tid] >> 6) != (s_key[tid - 1] >> 6));
            const unsigned bs = __ballot_sync(0xffffffffu, fs), bg = __ballot_sync(0xffffffffu, fg);
            if (lane == 0 && warp < nwr) { s_wcs[warp] = __popc(bs); s_wcg[warp] = __popc(bg); }
            __syncthreads();
            if (fs) {
                int before_s = 0, before_g = 0;
                for (int w = 0; w < warp; ++w) { before_s += s_wcs[w]; before_g += s_wcg[w]; }
                const unsigned lt = (1u << lane) - 1u;
                const int is = before_s + __popc(bs & lt);
                s_ss[is] = tid;
                if (fg) s_gss[before_g + __popc(bg & lt)] = is;
            }
            if (tid == 0) {
                int ts = 0, tg = 0;
                for (int w = 0; w < nwr; ++w) { ts += s_wcs[w]; tg += s_wcg[w]; }
                s_ss[ts] = n;
                s_gss[tg] = ts;
                s_ng = tg;
            }
            __syncthreads();
            const int nunits = s_ng * passes;

            // ---- units: (group, pass) with the lane's tap values in registers
            // tap of this lane in pass p: row jy = warp + (q / S) M, column q mod S, q = 32 p + lane
            auto tap_of = [&](int p, int &t, int &ct) {
                const int q = p * 32 + lane;
                const int lr = q / S;
                const int tx = q - lr * S, ty = warp + lr * M;
                t = (ty < S) ? ty * S + tx : -1;
                ct = ty * RS + tx;
            };
            auto load_unit = [&](int u, float2 (&k)[P]) {
                const int g = u / passes;
                int t, ct;
                tap_of(u - g * passes, t, ct);
                if (t >= 0) {
                    const int64_t kb = tab0 + (int64_t)(s_key[s_ss[s_gss[g]]] >> 6) * L * P;
                    if (RG_BOK(kb >= 0 && kb + (int64_t)P * L <= a.tab_elems, BC_R_TAB)) {
                        if constexpr (NPOL == 4) RgK<ST>::load(a.ktab, kb, L, t, k);
                        else k[0] = rg_k1<ST>(a.ktab, kb, t);
                    }
                }
            };
            auto run_unit = [&](int u, const float2 (&k)[P]) {
                const int g = u / passes;
                int t, ct;
                tap_of(u - g * passes, t, ct);
                const bool act = t >= 0;
                const int sg1 = s_gss[g + 1];
                for (int sg = s_gss[g]; sg < sg1; ++sg) {
                    const int j1 = s_ss[sg + 1];
                    for (int j = s_ss[sg]; j < j1; ++j) {
                        const int cell = s_cell[j] + ct;
                        if (act && RG_BOK(cell >= 0 && cell < RR, BC_R_SMEM)) {
                            if constexpr (NPOL == 1) {
                                const float2 v = s_v1[j];
                                float2 r = reg0[cell];
                                cmac2(r.x, r.y, k[0], v.x, v.y);
                                reg0[cell] = r;
                            } else {
                                float4 r01 = reg01[cell], r23 = reg23[cell];
                                mueller_acc(r01, r23, k, s_v[2 * j], s_v[2 * j + 1]);
                                reg01[cell] = r01;
                                reg23[cell] = r23;
                            }
                        }
                        // the next visibility's cells may be this one's cells of
                        // other lanes: its region reads come after these writes
                        __syncwarp();
                    }
                    // another footprint-row residue next: other warps may then
                    // write rows this warp wrote
                    __syncthreads();
                }
            };
            if constexpr (NPOL == 1) {
                const int tpl = passes;   // taps a lane: q = lane + 32 i, i < tpl, of (S / M) S
                const int tw = (S / M) * S;
                for (int g = 0; g < s_ng; ++g) {
                    float2 k[TMAX];
                    int ct[TMAX];
                    const int64_t kb = tab0 + (int64_t)(s_key[s_ss[s_gss[g]]] >> 6) * L;
                    const bool kok = RG_BOK(kb >= 0 && kb + (int64_t)L <= a.tab_elems, BC_R_TAB);
#pragma unroll
                    for (int i = 0; i < TMAX; ++i) {
                        const int q = lane + 32 * i;
                        const int lr = q / S, tx = q - lr * S, ty = warp + lr * M;
                        const bool on = i < tpl && q < tw && kok;
                        ct[i] = on ? ty * RS + tx : -1;
                        k[i] = on ? rg_k1<ST>(a.ktab, kb, ty * S + tx) : make_float2(0.f, 0.f);
                    }
                    const int sg1 = s_gss[g + 1];
                    for (int sg = s_gss[g]; sg < sg1; ++sg) {
                        const int j1 = s_ss[sg + 1];
                        for (int j = s_ss[sg]; j < j1; ++j) {
                            const int base = s_cell[j];
                            const float2 v = s_v1[j];
#pragma unroll
                            for (int i = 0; i < TMAX; ++i) {
                                const int cell = base + ct[i];
                                if (ct[i] >= 0 && RG_BOK(cell >= 0 && cell < RR, BC_R_SMEM)) {
                                    float2 r = reg0[cell];
                                    cmac2(r.x, r.y, k[i], v.x, v.y);
                                    reg0[cell] = r;
                                }
                            }
                            // the next visibility's cells may be this one's cells of other lanes
                            __syncwarp();
                        }
                        // another footprint-row residue next: other warps may then write rows this warp wrote
                        __syncthreads();
                    }
                }
            } else if constexpr (TMAX >= 2) {
                // TMAX passes of one offset group at a time: all their taps' cells are
                // read before any is written (distinct taps, distinct cells)
                for (int g = 0; g < s_ng; ++g) {
                    for (int p0 = 0; p0 < passes; p0 += TMAX) {
                        float2 kk[TMAX][P];
                        int tt[TMAX], ct[TMAX];
#pragma unroll
                        for (int i = 0; i < TMAX; ++i) {
#pragma unroll
                            for (int m = 0; m < P; ++m) kk[i][m] = make_float2(0.f, 0.f);
                            tt[i] = -1;
                            ct[i] = 0;
                            if (p0 + i < passes) {
                                load_unit(g * passes + p0 + i, kk[i]);
                                tap_of(p0 + i, tt[i], ct[i]);
                            }
                        }
                        const int sg1 = s_gss[g + 1];
                        for (int sg = s_gss[g]; sg < sg1; ++sg) {
                            const int j1 = s_ss[sg + 1];
                            for (int j = s_ss[sg]; j < j1; ++j) {
                                const int base = s_cell[j];
                                const float4 v01 = s_v[2 * j], v23 = s_v[2 * j + 1];
                                float4 c01[TMAX], c23[TMAX];
                                bool on[TMAX];
#pragma unroll
                                for (int i = 0; i < TMAX; ++i) {
                                    const int c = base + ct[i];
                                    on[i] = tt[i] >= 0 && RG_BOK(c >= 0 && c < RR, BC_R_SMEM);
                                    c01[i] = on[i] ? reg01[c] : z4;
                                    c23[i] = on[i] ? reg23[c] : z4;
                                }
#pragma unroll
                                for (int i = 0; i < TMAX; ++i) mueller_acc(c01[i], c23[i], kk[i], v01, v23);
#pragma unroll
                                for (int i = 0; i < TMAX; ++i)
                                    if (on[i]) {
                                        reg01[base + ct[i]] = c01[i];
                                        reg23[base + ct[i]] = c23[i];
                                    }
                                // the next visibility's cells may be this one's cells of other lanes
                                __syncwarp();
                            }
                            // another footprint-row residue next: other warps may then write rows this warp wrote
                            __syncthreads();
                        }
                    }
                }
            } else {
                for (int u = 0; u < nunits; ++u) {
                    float2 kA[P];
#pragma unroll
                    for (int m = 0; m < P; ++m) kA[m] = make_float2(0.f, 0.f);
                    load_unit(u, kA);
                    run_unit(u, kA);
                }
            }
        }
        __syncthreads();
        // ---- add the region to the grid (cells that received nothing are skipped)
        for (int c = tid; c < RR; c += BT) {
            const int cy = c / RS, cx = c - cy * RS;
            if (cx >= R) continue;   // row padding
            const int gy = oy + cy, gx = ox + cx;
            if constexpr (NPOL == 1) {
                const float2 v = reg0[c];
                if ((v.x != 0.f || v.y != 0.f) && RG_BOK(gy < a.N && gx < a.N, BC_R_GRID))
                    atomicAdd(a.grid + (int64_t)gy * a.N + gx, v);
                continue;
            }
            const float4 v01 = reg01[c], v23 = reg23[c];
            const bool nz = v01.x != 0.f || v01.y != 0.f || v01.z != 0.f || v01.w != 0.f ||
                            v23.x != 0.f || v23.y != 0.f || v23.z != 0.f || v23.w != 0.f;
            if (nz && RG_BOK(gy < a.N && gx < a.N, BC_R_GRID)) {
                float2 *dst = a.grid + (int64_t)gy * a.N + gx;
                atomicAdd(dst, make_float2(v01.x, v01.y));
                atomicAdd(dst + plane, make_float2(v01.z, v01.w));
                atomicAdd(dst + 2 * plane, make_float2(v23.x, v23.y));
                atomicAdd(dst + 3 * plane, make_float2(v23.z, v23.w));
            }
        }
    }
    // statistics: one atomic per CTA
    for (int o = 16; o; o >>= 1) {
        wloc += __shfl_xor_sync(0xffffffffu, wloc, o);
        nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    }
    if (lane == 0) { s_red[warp] = wloc; s_redn[warp] = nbad; }
    __syncthreads();
    if (tid == 0) {
        double tw = 0.0;
        unsigned long long tn = 0;
        for (int w = 0; w < BT / 32; ++w) { tw += s_red[w]; tn += s_redn[w]; }
        atomicAdd(a.wsum, tw);
        if (tn) atomicAdd(a.nonfinite, tn);
    }
}

template <int ST, int NPOL, int TMAX>
int launch_region_t(const RegionArgs &a, int BT, int sm_count, cudaStream_t s) {
    static_assert(AW_RG_RMAX <= 64, "region side");
    if (a.R != AW_RG_RMAX) return aw_set_error(AW_EINVAL, "region side %d", a.R);
    if (NPOL == 1 && (a.passes > TMAX || (BT != 64 && BT != 128)))
        return aw_set_error(AW_EINVAL, "Stokes-I region: %d taps a lane, %d threads", a.passes, BT);
    if (NPOL == 4 && TMAX >= 2 && BT > (TMAX == 3 ? 192 : 256))
        return aw_set_error(AW_EINVAL, "grouped region units: %d threads", BT);
    auto kern = grid_region_kernel<ST, AW_RG_RMAX, NPOL, TMAX>;
    const size_t smem = region_smem_bytes(a.R, NPOL);
    AW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    AW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, smem));
    int64_t blocks = std::min<int64_t>(a.nitems, (int64_t)sm_count * std::max(per_sm, 1));
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, BT, smem, s>>>(a);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

template <int TMAX>
int launch_region4(const RegionArgs &a, int st, int BT, int sm_count, cudaStream_t s) {
    if (st == AW_STORAGE_FP32) return launch_region_t<AW_STORAGE_FP32, 4, TMAX>(a, BT, sm_count, s);
    if (st == AW_STORAGE_BF16) return launch_region_t<AW_STORAGE_BF16, 4, TMAX>(a, BT, sm_count, s);
    return launch_region_t<AW_STORAGE_FP16, 4, TMAX>(a, BT, sm_count, s);
}

template <int TMAX>
int launch_region1(const RegionArgs &a, int st, int BT, int sm_count, cudaStream_t s) {
    if (st == AW_STORAGE_FP32) return launch_region_t<AW_STORAGE_FP32, 1, TMAX>(a, BT, sm_count, s);
    if (st == AW_STORAGE_BF16) return launch_region_t<AW_STORAGE_BF16, 1, TMAX>(a, BT, sm_count, s);
    return launch_region_t<AW_STORAGE_FP16, 1, TMAX>(a, BT, sm_count, s);
}

}  // namespace

int aw_region_rows(int S) {
    // row classes M (= warps of the CTA, 4..10) dividing S whose passes of 32
    // taps (S / M rows of S taps per warp) leave the fewest idle lanes; ties go
    // to more warps, except that a support done in one pass takes half the
    // warps, so that its units pair two passes (S = 16: 4 warps, 0.9 ms faster
    // on the 64M-visibility full-pol set than 8 warps in one pass; S = 40 keeps
    // 10 warps unpaired, 2.4 ms faster than 5 warps paired and 1.7 ms faster
    // than 8 warps paired).  0: none
    int best = 0;
    double best_eff = 0.0;
    for (int M = 10; M >= 4; --M) {
        if (S % M) continue;
        const int taps = (S / M) * S, passes = (taps + 31) / 32;
        const double eff = (double)taps / (32.0 * passes);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = M; }
    }
    if (best_eff < 0.74) return 0;
    if ((S / best) * S <= 32 && best / 2 >= 4 && S % (best / 2) == 0 && (S / (best / 2)) * S % 32 == 0) best /= 2;
    return best;
}

// Stokes I: 4 warps (row classes) for supports that are multiples of 4 and
// leave a lane at most RG_TPL1 taps; 0 if none.  (Measured on the 20.16M-
// visibility Stokes-I w-projection set: 4 warps 7.9 ms, 2 warps with twice the
// taps a lane 10.2 ms, 8-10 warps with one tap a lane 12.8 ms.)
static int region1_rows(int S) { return S >= 8 && S % 4 == 0 && ((S / 4) * S + 31) / 32 <= RG_TPL1 ? 4 : 0; }

int aw_region_tile(int S, int npol) {
    if (npol == 4 ? (S < 2 || aw_region_rows(S) == 0) : (npol != 1 || region1_rows(S) == 0)) return 0;
    const int T = AW_RG_RMAX - S + 1;
    return T >= 8 ? T : 0;
}

int aw_region_threads(int S, int npol) { return 32 * (npol == 1 ? region1_rows(S) : aw_region_rows(S)); }

int aw_launch_grid_region(const aw_plan *p, const aw_kernel_set *k, const void *vis, const float *weight, void *grid,
                          cudaStream_t s) {
    RegionArgs a;
    a.rec = p->d_rec_rg;
    a.ktab = k->d_table;
    a.bin_offset = k->d_bin_offset;
    a.bin_support = k->d_bin_support;
    a.vis = reinterpret_cast<const float2 *>(vis);
    a.weight = weight;
    a.grid = reinterpret_cast<float2 *>(grid);
    a.N = p->N;
    a.OS = p->OS;
    a.wsum = p->d_wsum;
    a.nonfinite = p->d_nonfinite;
    a.inv_scale = 1.0f / k->scale;
    a.nvis = p->nvis;
    a.nvalid = p->nreg;
    a.tab_elems = k->total_elems;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    AW_CUDA_TRY(cudaMemsetAsync(p->d_rcounter, 0, sizeof(unsigned int) * AW_RG_MAXCLASS, s));
    for (size_t i = 0; i < p->rclasses.size(); ++i) {
        const aw_plan::RegionClass &rc = p->rclasses[i];
        if (rc.n == 0) continue;
        a.items = rc.d_items;
        a.nitems = rc.n;
        a.counter = p->d_rcounter + i;
        a.S = rc.S;
        a.T = rc.T;
        a.R = rc.T + rc.S - 1;
        a.M = rc.BT / 32;
        a.passes = ((rc.S / a.M) * rc.S + 31) / 32;
        int r;
        const int st = k->spec.storage;
        if (p->npol == 4 && a.passes == 3 && rc.BT <= 192) {
            r = launch_region4<3>(a, st, rc.BT, sms, s);
        } else if (p->npol == 4 && a.passes >= 2 && rc.BT <= 256) {
            r = launch_region4<2>(a, st, rc.BT, sms, s);
        } else if (p->npol == 4) {
            r = launch_region4<1>(a, st, rc.BT, sms, s);
        } else if (a.passes <= 2) {
            r = launch_region1<2>(a, st, rc.BT, sms, s);
        } else if (a.passes <= 8) {
            r = launch_region1<8>(a, st, rc.BT, sms, s);
        } else {
            r = launch_region1<RG_TPL1>(a, st, rc.BT, sms, s);
        }
        if (r) return r;
    }
    return AW_OK;
}

int aw_region_bounds_status(unsigned int *v, int reset) {
#ifdef AW_BOUNDS_CHECK
    AW_CUDA_TRY(cudaMemcpyFromSymbol(v, g_bounds_status_rg, sizeof(*v)));
    if (reset) {
        const unsigned int z = 0;
        AW_CUDA_TRY(cudaMemcpyToSymbol(g_bounds_status_rg, &z, sizeof(z)));
    }
#else
    (void)reset;
    *v = 0;
#endif
    return AW_OK;
}
