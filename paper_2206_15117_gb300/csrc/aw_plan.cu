// Plan creation: per-visibility FP64 coordinates (uvw in wavelengths, Eq. 2)
// and the device key sort that orders visibilities by (bin, grid tile,
// position in tile) and cuts them into work items.
#include <algorithm>
#include <cmath>
#include <vector>

#include "aw_internal.h"

namespace {

struct CoordArgs {
    int64_t nvis;
    const double *uvw;
    const uint32_t *row;
    const uint16_t *chan;
    const double *freq;
    const uint8_t *pa_bin;
    const uint8_t *fbin;
    const uint8_t *flags;
    const uint8_t *row_types;  // [nrow][2] or NULL
    int N, OS, nw, npa, nfb, ntype;
    double uscale, half, winv;
    const int32_t *support;  // per w plane
    int tile, tbits, ntx, nty;
    int64_t nrow;
    int32_t nchan;
};

struct CoordOut {
    int x0, y0, fx, fy, bin, flip, valid, S;
};

// The FP64 coordinate step with a fixed operation order (no contraction).
__device__ __forceinline__ CoordOut coord_of(const CoordArgs &a, int64_t k) {
    CoordOut o;
    const uint32_t r = a.row[k];
    const uint16_t c = a.chan[k];
    const double f = __ddiv_rn(a.freq[c], AW_C_LIGHT);
    double u = __dmul_rn(a.uvw[3 * (int64_t)r + 0], f);
    double v = __dmul_rn(a.uvw[3 * (int64_t)r + 1], f);
    double w = __dmul_rn(a.uvw[3 * (int64_t)r + 2], f);
    o.flip = 0;
    if (w < 0.0) { u = -u; v = -v; w = -w; o.flip = 1; }
    const double xr = __dadd_rn(__dadd_rn(__dmul_rn(u, a.uscale), a.half), 0.5);
    const double yr = __dadd_rn(__dadd_rn(__dmul_rn(v, a.uscale), a.half), 0.5);
    // clamp far-out values before the integer conversion; they are invalid anyway
    const double lim = 4.0e15;
    const long long Xi = (long long)floor(fmin(fmax(xr, -lim), lim));
    const long long Yi = (long long)floor(fmin(fmax(yr, -lim), lim));
    int wp = 0;
    if (a.winv > 0.0) {
        const double wt = __dmul_rn(w, a.winv);
        const double fw = floor(fmin(wt, 1.0e9));
        wp = (int)fw;
        if (wp < 0) wp = 0;
        if (wp > a.nw - 1) wp = a.nw - 1;
    }
    const int pa = a.pa_bin ? (int)a.pa_bin[r] : 0;
    const int fb = a.fbin ? (int)a.fbin[c] : 0;
    int cls = 0;
    if (a.ntype >= 2 && a.row_types) {
        // the flipped sample is the reversed baseline: its class swaps the types
        int ti = min((int)a.row_types[2 * (int64_t)r], a.ntype - 1);
        int tj = min((int)a.row_types[2 * (int64_t)r + 1], a.ntype - 1);
        if (o.flip) { const int t = ti; ti = tj; tj = t; }
        cls = ti * a.ntype + tj;
    }
    o.bin = ((cls * a.nw + wp) * a.npa + min(pa, a.npa - 1)) * a.nfb + min(fb, a.nfb - 1);
    const int S = a.support[wp];
    o.S = S;
    const long long rho = (long long)(S - 2) * a.OS / 2;
    const long long Ax = Xi - rho, Ay = Yi - rho;
    long long ix = Ax / a.OS; if (Ax < 0 && ix * a.OS != Ax) ix -= 1;
    long long iy = Ay / a.OS; if (Ay < 0 && iy * a.OS != Ay) iy -= 1;
    o.fx = (int)(Ax - ix * a.OS);
    o.fy = (int)(Ay - iy * a.OS);
    int valid = 1;
    if (ix < 0 || ix + S > a.N) valid = 0;
    if (iy < 0 || iy + S > a.N) valid = 0;
    o.x0 = valid ? (int)ix : 0;
    o.y0 = valid ? (int)iy : 0;
    o.valid = valid;
    return o;
}

__global__ void coords_kernel(CoordArgs a, uint64_t invalid_key, uint64_t *keys, uint32_t *vals,
                              aw_rec *recs, unsigned long long *counts /* outside, flagged, valid, taps */) {
    unsigned long long n_out = 0, n_flag = 0, n_val = 0, taps = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.nvis;
         k += (int64_t)gridDim.x * blockDim.x) {
        const CoordOut o = coord_of(a, k);
        const bool flagged = a.flags && a.flags[k];
        const bool ok = o.valid && !flagged;
        if (!o.valid) n_out++;
        else if (flagged) n_flag++;
        uint64_t key = invalid_key;
        if (ok) {
            n_val++;
            taps += (unsigned long long)o.S * o.S;
            const int tx = o.x0 >> a.tbits, ty = o.y0 >> a.tbits;
            const int lx = o.x0 & (a.tile - 1), ly = o.y0 & (a.tile - 1);
            key = ((((uint64_t)o.bin * a.nty + ty) * a.ntx + tx) << (2 * a.tbits)) |
                  ((uint64_t)ly << a.tbits) | (uint64_t)lx;
        }
        keys[k] = key;
        vals[k] = (uint32_t)k;
        aw_rec rc;
        rc.orig = (uint32_t)k;
        rc.x0 = (uint16_t)o.x0;
        rc.y0 = (uint16_t)o.y0;
        rc.bin = (uint16_t)o.bin;
        rc.fx = (uint8_t)o.fx;
        rc.fy = (uint8_t)o.fy;
        rc.flip = (uint8_t)o.flip;
        rc.pad0 = ok ? 1 : 0;   // gridded
        rc.pad1 = 0;
        recs[k] = rc;
    }
    // warp-aggregated counters
    for (int off = 16; off; off >>= 1) {
        n_out += __shfl_xor_sync(0xffffffffu, n_out, off);
        n_flag += __shfl_xor_sync(0xffffffffu, n_flag, off);
        n_val += __shfl_xor_sync(0xffffffffu, n_val, off);
        taps += __shfl_xor_sync(0xffffffffu, taps, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_out) atomicAdd(&counts[0], n_out);
        if (n_flag) atomicAdd(&counts[1], n_flag);
        if (n_val) atomicAdd(&counts[2], n_val);
        if (taps) atomicAdd(&counts[3], taps);
    }
}

__global__ void coords_out_kernel(CoordArgs a, int32_t *x0, int32_t *y0, int32_t *fx, int32_t *fy,
                                  int32_t *bin, uint8_t *flip, uint8_t *valid) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.nvis;
         k += (int64_t)gridDim.x * blockDim.x) {
        const CoordOut o = coord_of(a, k);
        const bool ok = o.valid && !(a.flags && a.flags[k]);
        if (x0) x0[k] = o.x0;
        if (y0) y0[k] = o.y0;
        if (fx) fx[k] = o.fx;
        if (fy) fy[k] = o.fy;
        if (bin) bin[k] = o.bin;
        if (flip) flip[k] = (uint8_t)o.flip;
        if (valid) valid[k] = ok ? 1 : 0;
    }
}

// ------------------------------------------------------------ LSD radix sort
// One pass = per-tile digit histogram -> exclusive scan over [digit][tile] ->
// stable scatter.  A tile is RS_THREADS * RS_ITEMS keys; each warp owns a
// contiguous run of RS_ITEMS * 32 keys, ranks equal digits with
// __match_any_sync, and keeps its own running digit counters, so the order of
// equal keys is preserved.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void radix_hist_kernel(const uint64_t *keys, int64_t n, int shift, uint32_t *counts,
                                  int ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t k = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint64_t *keys, const uint32_t *vals, int64_t n, int shift,
                                     const uint32_t *offsets, int ntiles, uint64_t *keys_out,
                                     uint32_t *vals_out) {
    __shared__ uint32_t wbase[RS_WARPS][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wbase[0][0])[i] = 0;
    __syncthreads();
    const int64_t wstart = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_ITEMS * 32;
    uint64_t kk[RS_ITEMS];
    uint32_t vv[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t k = wstart + r * 32 + lane;
        kk[r] = (k < n) ? keys[k] : 0;
        vv[r] = (k < n) ? vals[k] : 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    // 1) per-warp digit counts
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t k = wstart + r * 32 + lane;
        const unsigned act = __ballot_sync(0xffffffffu, k < n);
        if (k < n) {
            const unsigned d = (unsigned)((kk[r] >> shift) & 0xFF);
            const unsigned peers = __match_any_sync(act, d);
            if ((peers & lt) == 0) wbase[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // 2) warp bases: global tile offset + counts of the earlier warps
    {
        const int d = threadIdx.x;  // RS_THREADS == 256 digits
        uint32_t run = offsets[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = wbase[w][d];
            wbase[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // 3) stable scatter, rounds in order
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t k = wstart + r * 32 + lane;
        const unsigned act = __ballot_sync(0xffffffffu, k < n);
        unsigned d = 0, peers = 0;
        uint32_t pos = 0;
        if (k < n) {
            d = (unsigned)((kk[r] >> shift) & 0xFF);
            peers = __match_any_sync(act, d);
            pos = wbase[warp][d] + __popc(peers & lt);
            keys_out[pos] = kk[r];
            vals_out[pos] = vv[r];
        }
        __syncwarp();
        if (k < n && (peers & lt) == 0) wbase[warp][d] += __popc(peers);
        __syncwarp();
    }
}

// ------------------------------------------------------------ items
__global__ void seg_flag_kernel(const uint64_t *keys, int64_t nvalid, int tb2, uint32_t *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvalid;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || (keys[i] >> tb2) != (keys[i - 1] >> tb2)) ? 1u : 0u;
}

__global__ void seg_start_kernel(const uint32_t *flag, const uint32_t *segid, int64_t nvalid,
                                 uint32_t *starts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvalid;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) starts[segid[i]] = (uint32_t)i;
}

__global__ void seg_chunks_kernel(const uint32_t *starts, int64_t nseg, uint32_t nvalid, int chunk,
                                  uint32_t *nch) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = starts[s];
        const uint32_t b = (s + 1 < nseg) ? starts[s + 1] : nvalid;
        nch[s] = (b - a + chunk - 1) / chunk;
    }
}

// bin_tile (may be NULL): per-bin region geometry (tile side in the low 8
// bits); then item.w holds the segment's tile as (row << 16) | column.
__global__ void emit_items_kernel(const uint32_t *starts, const uint32_t *itembase, int64_t nseg,
                                  uint32_t nvalid, int chunk, const aw_rec *rec, const int32_t *bin_tile,
                                  int4 *items) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = starts[s];
        const uint32_t b = (s + 1 < nseg) ? starts[s + 1] : nvalid;
        const aw_rec r = rec[a];
        const int bin = r.bin;
        int w = 0;
        if (bin_tile) {
            const int T = max(bin_tile[bin] & 0xff, 1);
            w = ((int)r.y0 / T) << 16 | ((int)r.x0 / T);
        }
        uint32_t pos = itembase[s];
        for (uint32_t st = a; st < b; st += chunk) {
            const uint32_t cnt = min((uint32_t)chunk, b - st);
            items[pos++] = make_int4((int)st, (int)cnt, bin, w);
        }
    }
}

// REGION key of the i-th valid visibility (grid order): (bin, region tile
// row, region tile column, oversampled offset, footprint row in the tile
// modulo M) above the position inside the tile (6 + 6 bits; tiles are at most
// 49 cells).  geo[bin] = T | M << 8 (0: the bin takes no region); those bins
// get invalid_key (sorted last); eligible ones are counted in *nreg.
__global__ void rg_key_kernel(const aw_rec *rec, int64_t nv, const int32_t *geo, int OS, int osb, int nt,
                              uint64_t invalid_key, uint64_t *keys, uint32_t *vals, unsigned long long *nreg) {
    unsigned long long cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const aw_rec r = rec[i];
        const int T = geo[r.bin] & 0xff, M = geo[r.bin] >> 8;
        uint64_t key = invalid_key;
        if (T > 0 && M > 0) {
            const int ty = (int)r.y0 / T, tx = (int)r.x0 / T;
            const int ly = (int)r.y0 - ty * T, lx = (int)r.x0 - tx * T;
            const uint64_t grp = ((((uint64_t)r.bin * nt + ty) * nt + tx) << osb) | (uint64_t)(r.fy * OS + r.fx);
            key = (((grp << 4) | (uint64_t)(ly % M)) << 12) | ((uint64_t)ly << 6) | (uint64_t)lx;
            cnt++;
        }
        keys[i] = key;
        vals[i] = (uint32_t)i;
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nreg, cnt);
}


__global__ void gather_rec_kernel(const aw_rec *in, const uint32_t *perm, int64_t n, aw_rec *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

__global__ void rec_orig_kernel(const aw_rec *rec, int64_t n, uint32_t *perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = rec[i].orig;
}

// Degridding key of the i-th valid visibility (grid order): (bin, super-tile
// row, super-tile column, fy, fx) above the position inside the super-tile.
__global__ void dg_key_kernel(const aw_rec *rec, int64_t nv, int OS, int stbits, int nst, uint64_t *keys,
                              uint32_t *vals) {
    const int smask = (1 << stbits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x) {
        const aw_rec r = rec[i];
        const uint64_t grp = (((uint64_t)r.bin * nst + (r.y0 >> stbits)) * nst + (r.x0 >> stbits)) * OS * OS +
                             (uint64_t)r.fy * OS + r.fx;
        keys[i] = (grp << (2 * stbits)) | ((uint64_t)(r.y0 & smask) << stbits) | (uint64_t)(r.x0 & smask);
        vals[i] = (uint32_t)i;
    }
}

int grid_blocks(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) aw_dev_free(p); }
};

int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

int fill_coord_args(const aw_vis_desc *vis, const aw_kernel_set *ks, int tile, CoordArgs &a,
                    aw_plan *plan) {
    const aw_kernel_spec &sp = ks->spec;
    a.nvis = vis->nvis;
    a.uvw = vis->uvw;
    a.row = vis->row_of_vis;
    a.chan = vis->chan_of_vis;
    a.freq = vis->freq;
    a.pa_bin = vis->pa_bin;
    a.fbin = vis->fbin;
    a.flags = vis->flags;
    a.row_types = vis->row_types;
    a.N = sp.N;
    a.OS = sp.OS;
    a.nw = sp.nw;
    a.npa = sp.npa;
    a.nfb = sp.nfb;
    a.ntype = ks->ntype;
    a.uscale = (double)sp.N * sp.dl * (double)sp.OS;
    a.half = (double)(sp.N / 2) * (double)sp.OS;
    a.winv = (sp.nw > 1 && sp.w_max > 0.0) ? (double)sp.nw / sp.w_max : 0.0;
    a.support = plan->d_plane_support;  // first nw entries hold the per-plane supports
    a.tile = tile;
    a.tbits = ilog2(tile);
    a.ntx = (sp.N + tile - 1) / tile;
    a.nty = a.ntx;
    a.nrow = vis->nrow;
    a.nchan = vis->nchan;
    return AW_OK;
}

// LSD radix sort of (key, value) pairs over `passes` 8-bit digits; on return
// k0/v0 point at the sorted arrays.  `counts`/`offs` hold 256 * ceil(n / RS_TILE)
// words, `scratch` serves the exclusive scan of that many words.
int radix_sort_pairs(uint64_t *&k0, uint32_t *&v0, uint64_t *&k1, uint32_t *&v1, int64_t n, int passes,
                     uint32_t *counts, uint32_t *offs, void *scratch, cudaStream_t s) {
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    const int64_t ncounts = (int64_t)256 * ntiles;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = pass * 8;
        radix_hist_kernel<<<ntiles, RS_THREADS, 0, s>>>(k0, n, shift, counts, ntiles);
        AW_CHECK_LAUNCH();
        int rc = aw_exclusive_scan_u32(counts, offs, ncounts, scratch, s);
        if (rc) return rc;
        radix_scatter_kernel<<<ntiles, RS_THREADS, 0, s>>>(k0, v0, n, shift, offs, ntiles, k1, v1);
        AW_CHECK_LAUNCH();
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    return AW_OK;
}

// Cut the sorted keys of the nv valid visibilities into segments of equal
// key >> shift and the segments into items of at most `chunk` visibilities;
// allocates *items.  `flag`/`segid` hold nv + 1 words each.
int build_items(const uint64_t *keys, int64_t nv, int shift, int chunk, const aw_rec *rec, uint32_t *flag,
                uint32_t *segid, void *scratch, int4 **items, int64_t *nitems, cudaStream_t s,
                const int32_t *bin_tile = nullptr) {
    seg_flag_kernel<<<grid_blocks(nv, 256), 256, 0, s>>>(keys, nv, shift, flag);
    AW_CHECK_LAUNCH();
    int rc = aw_exclusive_scan_u32(flag, segid, nv, scratch, s);
    if (rc) return rc;
    uint32_t last_id = 0, last_flag = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&last_id, segid + nv - 1, 4, cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaMemcpyAsync(&last_flag, flag + nv - 1, 4, cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nseg = (int64_t)last_id + last_flag;
    DevBuf bstarts, bnch, bbase;
    AW_CUDA_TRY(aw_dev_malloc(&bstarts.p, sizeof(uint32_t) * nseg));
    AW_CUDA_TRY(aw_dev_malloc(&bnch.p, sizeof(uint32_t) * nseg));
    AW_CUDA_TRY(aw_dev_malloc(&bbase.p, sizeof(uint32_t) * nseg));
    seg_start_kernel<<<grid_blocks(nv, 256), 256, 0, s>>>(flag, segid, nv, (uint32_t *)bstarts.p);
    AW_CHECK_LAUNCH();
    seg_chunks_kernel<<<grid_blocks(nseg, 256), 256, 0, s>>>((uint32_t *)bstarts.p, nseg, (uint32_t)nv, chunk,
                                                            (uint32_t *)bnch.p);
    AW_CHECK_LAUNCH();
    rc = aw_exclusive_scan_u32((uint32_t *)bnch.p, (uint32_t *)bbase.p, nseg, scratch, s);
    if (rc) return rc;
    uint32_t lb = 0, ln = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&lb, (uint32_t *)bbase.p + nseg - 1, 4, cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaMemcpyAsync(&ln, (uint32_t *)bnch.p + nseg - 1, 4, cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    *nitems = (int64_t)lb + ln;
    AW_CUDA_TRY(aw_dev_malloc(items, sizeof(int4) * std::max<int64_t>(*nitems, 1)));
    emit_items_kernel<<<grid_blocks(nseg, 256), 256, 0, s>>>((uint32_t *)bstarts.p, (uint32_t *)bbase.p, nseg,
                                                            (uint32_t)nv, chunk, rec, bin_tile, *items);
    AW_CHECK_LAUNCH();
    // the temporaries are freed on return: finish the kernels that read them
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    return AW_OK;
}

}  // namespace

// AW_GRID_HYBRID: the gridding items of w planes [0, split_planes) for the
// TILES part and the degridding items of the other planes for the OFFSETS
// part (order kept), plus the second stream and the fork / join events.  The
// w plane of bin ((k nw + p) npa + a) nfb + f is p.  Once per plan, on the host.
static int build_hybrid_items(aw_plan *plan, cudaStream_t s) {
    const int split = plan->tune.split_planes, per_plane = plan->npa * plan->nfb;
    auto filter = [&](const int4 *d_src, int64_t n, bool low, int4 **d_out, int64_t *n_out) -> int {
        std::vector<int4> h((size_t)n), keep;
        if (n) AW_CUDA_TRY(cudaMemcpyAsync(h.data(), d_src, sizeof(int4) * n, cudaMemcpyDeviceToHost, s));
        AW_CUDA_TRY(cudaStreamSynchronize(s));
        keep.reserve((size_t)n);
        for (const int4 &it : h)
            if (((it.z / per_plane) % plan->nw < split) == low) keep.push_back(it);
        *n_out = (int64_t)keep.size();
        if (!keep.empty()) {
            AW_CUDA_TRY(aw_dev_malloc(d_out, sizeof(int4) * keep.size()));
            AW_CUDA_TRY(cudaMemcpyAsync(*d_out, keep.data(), sizeof(int4) * keep.size(), cudaMemcpyHostToDevice, s));
            AW_CUDA_TRY(cudaStreamSynchronize(s));
        }
        return AW_OK;
    };
    int rc = filter(plan->d_items, plan->nitems, true, &plan->d_items_ht, &plan->nitems_ht);
    if (rc) return rc;
    rc = filter(plan->d_items_dg, plan->nitems_dg, false, &plan->d_items_ho, &plan->nitems_ho);
    if (rc) return rc;
    AW_CUDA_TRY(cudaStreamCreateWithFlags(&plan->aux, cudaStreamNonBlocking));
    AW_CUDA_TRY(cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming));
    AW_CUDA_TRY(cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming));
    return AW_OK;
}

// AW_GRID_REGION: the region order of the valid visibilities of bins whose
// support fits a region (aw_region_tile), its items bucketed by support (one
// launch each), and the OFFSETS items of the other bins with the second
// stream.  k0/v0/k1/v1 and the scan buffers are the plan builder's (>= nv).
static int build_region(aw_plan *plan, const aw_kernel_set *ks, int64_t nv, uint64_t *k0, uint32_t *v0,
                        uint64_t *k1, uint32_t *v1, uint32_t *counts, uint32_t *offs, void *scratch,
                        cudaStream_t s) {
    const int nb = ks->nbins;
    std::vector<int32_t> bt((size_t)nb, 0);
    // bins of w planes [0, split_planes) (all planes when 0) whose support fits a region
    const int per_plane = plan->npa * plan->nfb;
    const int split = plan->tune.split_planes > 0 ? plan->tune.split_planes : plan->nw;
    for (int b = 0; b < nb; ++b) {
        const int S = ks->bin_support[(size_t)b], T = aw_region_tile(S, plan->npol);
        const bool low = (b / per_plane) % plan->nw < split;
        bt[(size_t)b] = (T && low) ? (T | aw_region_threads(S, plan->npol) / 32 << 8) : 0;
    }
    DevBuf dbt, dcnt;
    AW_CUDA_TRY(aw_dev_malloc(&dbt.p, sizeof(int32_t) * std::max(nb, 1)));
    AW_CUDA_TRY(cudaMemcpyAsync(dbt.p, bt.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
    AW_CUDA_TRY(aw_dev_malloc(&dcnt.p, sizeof(unsigned long long)));
    AW_CUDA_TRY(cudaMemsetAsync(dcnt.p, 0, sizeof(unsigned long long), s));
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_rcounter, sizeof(unsigned int) * AW_RG_MAXCLASS));
    const int OS = plan->OS;
    const int osb = ilog2(OS * OS);
    const int nt = (plan->N + 7) / 8;
    const uint64_t maxgrp = ((uint64_t)nb * nt * nt) << osb;
    int gbits = 0;
    while (gbits < 63 && (1ull << gbits) <= maxgrp) ++gbits;
    if (gbits + 16 > 62) return aw_set_error(AW_EINVAL, "region key needs %d bits", gbits + 16);
    const int kbits = gbits + 16;
    const uint64_t invalid_key = 1ull << kbits;
    rg_key_kernel<<<grid_blocks(nv, 256), 256, 0, s>>>(plan->d_rec, nv, (const int32_t *)dbt.p, OS, osb, nt,
                                                      invalid_key, k0, v0, (unsigned long long *)dcnt.p);
    AW_CHECK_LAUNCH();
    int rc = radix_sort_pairs(k0, v0, k1, v1, nv, (kbits + 1 + 7) / 8, counts, offs, scratch, s);
    if (rc) return rc;
    unsigned long long nreg = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&nreg, dcnt.p, sizeof(nreg), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    plan->nreg = (int64_t)nreg;
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_rec_rg, sizeof(aw_rec) * std::max<int64_t>(plan->nreg, 1)));
    if (plan->nreg > 0) {
        gather_rec_kernel<<<grid_blocks(plan->nreg, 256), 256, 0, s>>>(plan->d_rec, v0, plan->nreg, plan->d_rec_rg);
        AW_CHECK_LAUNCH();
        int4 *d_items = nullptr;
        int64_t nitems = 0;
        rc = build_items(k0, plan->nreg, osb + 16, AW_RG_MAXV, plan->d_rec_rg, counts, offs, scratch, &d_items,
                         &nitems, s, (const int32_t *)dbt.p);
        if (rc) return rc;
        std::vector<int4> h((size_t)nitems);
        cudaError_t e = cudaMemcpyAsync(h.data(), d_items, sizeof(int4) * nitems, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        aw_dev_free(d_items);
        if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "region items: %s", cudaGetErrorString(e));
        // one list per support, in increasing support (order inside a list kept)
        std::map<int, std::vector<int4>> by_s;
        for (const int4 &it : h) by_s[ks->bin_support[(size_t)it.z]].push_back(it);
        if ((int)by_s.size() > AW_RG_MAXCLASS) return aw_set_error(AW_EUNSUPPORTED, "%d supports", (int)by_s.size());
        for (auto &kv : by_s) {
            aw_plan::RegionClass c;
            c.S = kv.first;
            c.T = aw_region_tile(c.S, plan->npol);
            c.BT = aw_region_threads(c.S, plan->npol);
            c.n = (int64_t)kv.second.size();
            plan->rclasses.push_back(c);
            AW_CUDA_TRY(aw_dev_malloc(&plan->rclasses.back().d_items, sizeof(int4) * kv.second.size()));
            AW_CUDA_TRY(cudaMemcpyAsync(plan->rclasses.back().d_items, kv.second.data(), sizeof(int4) * kv.second.size(),
                                        cudaMemcpyHostToDevice, s));
        }
    }
    // the other bins: their degridding items on the OFFSETS schedule
    std::vector<int4> hd((size_t)plan->nitems_dg), keep;
    if (plan->nitems_dg)
        AW_CUDA_TRY(cudaMemcpyAsync(hd.data(), plan->d_items_dg, sizeof(int4) * plan->nitems_dg, cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    for (const int4 &it : hd)
        if (bt[(size_t)it.z] == 0) keep.push_back(it);
    plan->nitems_ho = (int64_t)keep.size();
    if (!keep.empty()) {
        AW_CUDA_TRY(aw_dev_malloc(&plan->d_items_ho, sizeof(int4) * keep.size()));
        AW_CUDA_TRY(cudaMemcpyAsync(plan->d_items_ho, keep.data(), sizeof(int4) * keep.size(), cudaMemcpyHostToDevice, s));
    }
    AW_CUDA_TRY(cudaStreamCreateWithFlags(&plan->aux, cudaStreamNonBlocking));
    AW_CUDA_TRY(cudaEventCreateWithFlags(&plan->ev_fork, cudaEventDisableTiming));
    AW_CUDA_TRY(cudaEventCreateWithFlags(&plan->ev_join, cudaEventDisableTiming));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    return AW_OK;
}

int aw_plan_plane_taps(const aw_plan *plan, std::vector<double> &cum, cudaStream_t s) {
    cum.assign((size_t)plan->nw + 1, 0.0);
    std::vector<int4> h((size_t)plan->nitems);
    if (plan->nitems) AW_CUDA_TRY(cudaMemcpyAsync(h.data(), plan->d_items, sizeof(int4) * plan->nitems,
                                                  cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    const int per_plane = plan->npa * plan->nfb;
    for (const int4 &it : h) {
        const double S = plan->bin_support[(size_t)it.z];
        cum[(size_t)((it.z / per_plane) % plan->nw) + 1] += (double)it.y * S * S;
    }
    for (size_t q = 1; q < cum.size(); ++q) cum[q] += cum[q - 1];
    if (cum.back() > 0)
        for (double &c : cum) c /= cum.back();
    return AW_OK;
}

int aw_plan_build(aw_ctx *ctx, const aw_vis_desc *vis, const aw_kernel_set *ks, const aw_tune *tune,
                  aw_plan *plan, cudaStream_t s) {
    (void)ctx;
    if (!vis || vis->nvis < 0 || (vis->nvis > 0 && (!vis->uvw || !vis->row_of_vis || !vis->chan_of_vis || !vis->freq)))
        return aw_set_error(AW_EINVAL, "vis descriptor incomplete");
    if (vis->nvis > 0x7fffffffLL) return aw_set_error(AW_EINVAL, "nvis %lld above 2^31-1", (long long)vis->nvis);
    const aw_kernel_spec &sp = ks->spec;
    aw_tune t = tune ? *tune : aw_tune{32, 256, 2, 0, AW_GRID_TILES};
    if (t.tile < 8 || t.tile > 256 || (t.tile & (t.tile - 1))) return aw_set_error(AW_EINVAL, "tile %d", t.tile);
    if (t.chunk < 32 || t.chunk > 2048) return aw_set_error(AW_EINVAL, "chunk %d", t.chunk);
    if (t.ctas_per_sm < 1 || t.ctas_per_sm > 8) t.ctas_per_sm = 2;
    if (t.dg_tile == 0) t.dg_tile = 1024;
    if (t.dg_tile < 32 || t.dg_tile > 4096 || (t.dg_tile & (t.dg_tile - 1)))
        return aw_set_error(AW_EINVAL, "dg_tile %d", t.dg_tile);
    if (t.grid_mode != AW_GRID_TILES && t.grid_mode != AW_GRID_OFFSETS && t.grid_mode != AW_GRID_HYBRID &&
        t.grid_mode != AW_GRID_REGION)
        return aw_set_error(AW_EINVAL, "grid_mode %d", t.grid_mode);
    if ((t.grid_mode == AW_GRID_HYBRID || t.grid_mode == AW_GRID_REGION) &&
        (t.split_planes < 0 || t.split_planes > sp.nw))
        return aw_set_error(AW_EINVAL, "split_planes %d outside 0..%d", t.split_planes, sp.nw);
    plan->tune = t;
    plan->dg_tile = t.dg_tile;
    plan->nvis = vis->nvis;
    plan->N = sp.N;
    plan->OS = sp.OS;
    plan->npol = sp.npol;
    plan->nbins = ks->nbins;
    plan->nw = sp.nw;
    plan->npa = sp.npa;
    plan->nfb = sp.nfb;
    plan->ntype = ks->ntype;
    plan->vis = *vis;
    // per-plane supports first (the coordinate step indexes by w plane), then per bin
    std::vector<int32_t> sup(ks->supports.begin(), ks->supports.end());
    plan->bin_support = ks->bin_support;
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_plane_support, sizeof(int32_t) * std::max<size_t>(sup.size(), 1)));
    AW_CUDA_TRY(cudaMemcpy(plan->d_plane_support, sup.data(), sizeof(int32_t) * sup.size(), cudaMemcpyHostToDevice));
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_wsum, sizeof(double)));
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_nonfinite, sizeof(unsigned long long)));
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_counter, sizeof(unsigned int) * 4));
    const int64_t n = vis->nvis;
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_rec, sizeof(aw_rec) * std::max<int64_t>(n, 1)));
    if (n == 0) {
        AW_CUDA_TRY(aw_dev_malloc(&plan->d_items, sizeof(int4)));
        return AW_OK;
    }
    CoordArgs a;
    fill_coord_args(vis, ks, t.tile, a, plan);
    plan->uscale = a.uscale;
    plan->half = a.half;
    plan->winv = a.winv;
    // key width: bins x tiles x (tile position), plus one bit for invalid
    const uint64_t maxkey = ((uint64_t)ks->nbins * a.nty * a.ntx) << (2 * a.tbits);
    int kbits = 0;
    while (kbits < 63 && (1ull << kbits) <= maxkey) ++kbits;
    const uint64_t invalid_key = 1ull << kbits;
    const int passes = (kbits + 1 + 7) / 8;

    DevBuf bk0, bk1, bv0, bv1, brec, bcnt, bcounts, bscan, bscratch;
    AW_CUDA_TRY(aw_dev_malloc(&bk0.p, sizeof(uint64_t) * n));
    AW_CUDA_TRY(aw_dev_malloc(&bk1.p, sizeof(uint64_t) * n));
    AW_CUDA_TRY(aw_dev_malloc(&bv0.p, sizeof(uint32_t) * n));
    AW_CUDA_TRY(aw_dev_malloc(&bv1.p, sizeof(uint32_t) * n));
    AW_CUDA_TRY(aw_dev_malloc(&brec.p, sizeof(aw_rec) * n));
    AW_CUDA_TRY(aw_dev_malloc(&bcnt.p, sizeof(unsigned long long) * 4));
    AW_CUDA_TRY(cudaMemsetAsync(bcnt.p, 0, sizeof(unsigned long long) * 4, s));
    uint64_t *k0 = (uint64_t *)bk0.p, *k1 = (uint64_t *)bk1.p;
    uint32_t *v0 = (uint32_t *)bv0.p, *v1 = (uint32_t *)bv1.p;
    coords_kernel<<<grid_blocks(n, 256), 256, 0, s>>>(a, invalid_key, k0, v0, (aw_rec *)brec.p,
                                                     (unsigned long long *)bcnt.p);
    AW_CHECK_LAUNCH();
    // radix sort passes
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    const int64_t ncounts = (int64_t)256 * ntiles;
    const int64_t scan_n = std::max<int64_t>(ncounts, n + 1);
    AW_CUDA_TRY(aw_dev_malloc(&bcounts.p, sizeof(uint32_t) * scan_n));
    AW_CUDA_TRY(aw_dev_malloc(&bscan.p, sizeof(uint32_t) * scan_n));
    AW_CUDA_TRY(aw_dev_malloc(&bscratch.p, aw_scan_scratch_bytes(scan_n)));
    uint32_t *counts = (uint32_t *)bcounts.p, *offs = (uint32_t *)bscan.p;
    int rc = radix_sort_pairs(k0, v0, k1, v1, n, passes, counts, offs, bscratch.p, s);
    if (rc) return rc;
    gather_rec_kernel<<<grid_blocks(n, 256), 256, 0, s>>>((aw_rec *)brec.p, v0, n, plan->d_rec);
    AW_CHECK_LAUNCH();
    unsigned long long hc[4];
    AW_CUDA_TRY(cudaMemcpyAsync(hc, bcnt.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    plan->n_outside = (int64_t)hc[0];
    plan->n_flagged = (int64_t)hc[1];
    plan->nvalid = (int64_t)hc[2];
    plan->mean_taps = hc[2] ? (double)hc[3] / (double)hc[2] : 0.0;
    const int64_t nv = plan->nvalid;
    if (nv == 0) {
        AW_CUDA_TRY(aw_dev_malloc(&plan->d_items, sizeof(int4)));
        plan->nitems = 0;
        return AW_OK;
    }
    // gridding items: runs of equal (bin, tile), then chunks
    rc = build_items(k0, nv, 2 * a.tbits, t.chunk, plan->d_rec, counts, offs, bscratch.p, &plan->d_items,
                     &plan->nitems, s);
    if (rc) return rc;

    // degridding order: (bin, super-tile, oversampled offset, position in super-tile)
    const int stbits = ilog2(plan->dg_tile);
    const int nst = (sp.N + plan->dg_tile - 1) >> stbits;
    const uint64_t ngroups = (uint64_t)ks->nbins * nst * nst * sp.OS * sp.OS;
    const uint64_t dg_maxkey = ngroups << (2 * stbits);
    int dg_bits = 0;
    while (dg_bits < 63 && (1ull << dg_bits) <= dg_maxkey) ++dg_bits;
    if (dg_bits > 62) return aw_set_error(AW_EINVAL, "degridding key needs %d bits; raise dg_tile", dg_bits);
    dg_key_kernel<<<grid_blocks(nv, 256), 256, 0, s>>>(plan->d_rec, nv, sp.OS, stbits, nst, k0, v0);
    AW_CHECK_LAUNCH();
    rc = radix_sort_pairs(k0, v0, k1, v1, nv, (dg_bits + 7) / 8, counts, offs, bscratch.p, s);
    if (rc) return rc;
    AW_CUDA_TRY(aw_dev_malloc(&plan->d_rec_dg, sizeof(aw_rec) * nv));
    gather_rec_kernel<<<grid_blocks(nv, 256), 256, 0, s>>>(plan->d_rec, v0, nv, plan->d_rec_dg);
    AW_CHECK_LAUNCH();
    rc = build_items(k0, nv, 2 * stbits, AW_DG_CHUNK, plan->d_rec_dg, counts, offs, bscratch.p,
                     &plan->d_items_dg, &plan->nitems_dg, s);
    if (rc) return rc;
    if (t.grid_mode == AW_GRID_HYBRID) {
        rc = build_hybrid_items(plan, s);
        if (rc) return rc;
    }
    if (t.grid_mode == AW_GRID_REGION) {
        rc = build_region(plan, ks, nv, k0, v0, k1, v1, counts, offs, bscratch.p, s);
        if (rc) return rc;
    }
    AW_CUDA_TRY(cudaStreamSynchronize(s));
    return AW_OK;
}

int aw_plan_coords_impl(const aw_plan *plan, const aw_kernel_set *ks_unused, int32_t *x0, int32_t *y0,
                        int32_t *fx, int32_t *fy, int32_t *bin, uint8_t *flip, uint8_t *valid,
                        cudaStream_t s) {
    (void)ks_unused;
    if (plan->nvis == 0) return AW_OK;
    CoordArgs a;
    const aw_vis_desc *vis = &plan->vis;
    a.nvis = vis->nvis;
    a.uvw = vis->uvw;
    a.row = vis->row_of_vis;
    a.chan = vis->chan_of_vis;
    a.freq = vis->freq;
    a.pa_bin = vis->pa_bin;
    a.fbin = vis->fbin;
    a.flags = vis->flags;
    a.row_types = vis->row_types;
    a.N = plan->N;
    a.OS = plan->OS;
    a.nw = plan->nw;
    a.npa = plan->npa;
    a.nfb = plan->nfb;
    a.ntype = plan->ntype;
    a.uscale = plan->uscale;
    a.half = plan->half;
    a.winv = plan->winv;
    a.support = plan->d_plane_support;
    a.tile = plan->tune.tile;
    a.tbits = ilog2(plan->tune.tile);
    a.ntx = a.nty = (plan->N + plan->tune.tile - 1) / plan->tune.tile;
    coords_out_kernel<<<grid_blocks(plan->nvis, 256), 256, 0, s>>>(a, x0, y0, fx, fy, bin, flip, valid);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

int aw_plan_order_impl(const aw_plan *plan, uint32_t *perm, cudaStream_t s) {
    if (plan->nvis == 0) return AW_OK;
    rec_orig_kernel<<<grid_blocks(plan->nvis, 256), 256, 0, s>>>(plan->d_rec, plan->nvis, perm);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

// ------------------------------------------------------------ exclusive scan
// Three phases over blocks of SCAN_BLOCK elements: block sums, a scan of the
// block sums by one block, then the block-local scan plus its offset.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_BLOCK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t ws = (lane < SCAN_THREADS / 32) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = ws;
    }
    __syncthreads();
    const uint32_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    if (total) *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void scan_reduce_kernel(const uint32_t *in, int64_t n, uint32_t *bsum) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(uint32_t *bsum, int64_t nb) {
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = (i < nb) ? bsum[i] : 0;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, &total);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void scan_apply_kernel(const uint32_t *in, int64_t n, const uint32_t *bsum, uint32_t *out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t run = block_exclusive_scan(s, nullptr) + bsum[blockIdx.x];
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

size_t aw_scan_scratch_bytes(int64_t n) {
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    return sizeof(uint32_t) * (size_t)std::max<int64_t>(nb, 1);
}

int aw_exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, void *scratch, cudaStream_t s) {
    if (n <= 0) return AW_OK;
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb > 0x7fffffffLL) return aw_set_error(AW_EINVAL, "scan too large");
    uint32_t *bsum = (uint32_t *)scratch;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
    AW_CHECK_LAUNCH();
    scan_sums_kernel<<<1, SCAN_THREADS, 0, s>>>(bsum, nb);
    AW_CHECK_LAUNCH();
    scan_apply_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum, out);
    AW_CHECK_LAUNCH();
    return AW_OK;
}
