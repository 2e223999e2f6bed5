// Training the learned kernel surrogate on the 5th-generation tensor cores.
//
// The network and its loss are the ones aw_mlp.cu defines (SIREN layers
// h = sin(omega0 (W h_prev + b)), linear output, L = (1/B) sum (y - t)^2; the
// kernels it learns are Sec. 3.2's uv transforms of the Mueller cells after the
// anti-aliasing function and the w term).  For a network of width 128 the
// large products of a training step run as tcgen05.mma (kind::f16: FP16
// operands, FP32 accumulators in tensor memory), the rest on the CUDA cores:
//
//   forward   layer 1 (5 inputs) on the CUDA cores; every further layer one
//             GEMM over 128-row tiles of the batch: Z = H_prev W^T + b, with
//             the epilogue writing H = sin(omega0 Z) (FP16) and cos(omega0 Z)
//             (FP16, all the backward pass needs of Z); the output layer's
//             epilogue forms the loss, dY = 2 (Y - T) and the output bias
//             gradient (the column sums of dY)
//   backward  dH_prev = dZ W (a GEMM with W^T as the K-major operand) whose
//             epilogue multiplies by omega0 cos(omega0 Z_prev); the weight
//             gradient dW = dZ^T H_prev as a GEMM whose K is the batch, split
//             over the SMs, accumulated in tensor memory and added to the FP32
//             gradient; dZ and H_prev enter it as they are stored (batch rows)
//             through the tensor cores' MN-major operand layout, and a hidden
//             layer's bias gradient (the column sums of dZ) rides in the same
//             GEMM as an extra operand column of ones; layer 1 on the CUDA cores
//
// The gradients are those of the summed loss times 1/B, i.e. of L itself, so
// Adam on the FP32 master parameters (aw_mlp.cu) is unchanged; after each
// step the FP16 copies of W and W^T used as operands are refreshed.  FP16
// operands keep 11 significand bits: the gradients match the FP64 oracle to
// about 1e-3 relative per layer.
//
// Operand tiles sit in shared memory without swizzle, in 8 x 8 core matrices
// of 128 bytes (8 rows of 16 contiguous bytes).  K-major (the per-layer
// GEMMs): the K-adjacent core matrices 128 B apart (LBO) and 8-row groups
// KT * 16 B apart (SBO, KT the K extent of the tile).  MN-major (the
// weight-gradient GEMMs): a core matrix holds 8 K-rows of 8 MN-elements, the
// MN-adjacent ones 128 B apart (SBO) and the K-adjacent ones X * 16 B apart
// (LBO, X the MN extent).  Each MMA takes K = 16.  The per-layer GEMMs run
// persistent, one CTA per SM over the batch's 128-row tiles with two operand
// stages and two accumulators; the weight-gradient GEMMs as one CTA per SM,
// each a slice of the batch, adding its partial product to the FP32 gradient
// atomically.  Every mbarrier wait is bounded; a wait that gives up records an
// error word the host reads after the step.
#include <algorithm>
#include <cmath>

#include "aw_mlp.h"

namespace {

constexpr int TCW = 128;                         // network width the tensor-core path takes
constexpr long long TC_WAIT_LIMIT = 1ll << 22;   // mbarrier polls (with back-off) before giving up

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major core-matrix tile whose K extent is KT
template <int KT>
__device__ __forceinline__ uint32_t cm(int r, int k) {
    return (uint32_t)(((r >> 3) * (KT / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30),
// SBO >> 4 [32,46), version 1 [46,48), no swizzle [61,64)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// shared-memory matrix descriptor with explicit LBO and SBO
__device__ __forceinline__ uint64_t sdesc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor, kind::f16: D F32 [4,6) = 1, A = B = F16, A and B
// K-major unless mn_a / mn_b (bits 15, 16: MN-major), N >> 3 at [17,23),
// M >> 4 at [24,29)
__host__ __device__ constexpr uint32_t idesc(int M, int N, int mn_a = 0, int mn_b = 0) {
    return (1u << 4) | ((uint32_t)mn_a << 15) | ((uint32_t)mn_b << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

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
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

// sin and cos of x: x reduced to about [-pi, pi] by subtracting k 2 pi in two
// parts (Cody and Waite's reduction: the head 201/32 has 8 significant bits, so
// k times it is exact for |k| < 2^16, and the tail carries the rest of 2 pi),
// then the special-function unit's approximations, which are accurate to a few
// 1e-7 absolute on that interval, for any |x| below about 4e5.
__device__ __forceinline__ void sincos_red(float x, float *sn, float *cs) {
    const float k = rintf(x * 0.15915494309189535f);
    float r = fmaf(-k, 6.28125f, x);                  // 6.28125 = 201 / 32
    r = fmaf(-k, 1.9353071795864769e-3f, r);          // 2 pi - 6.28125
    __sincosf(r, sn, cs);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// rows [r0, r0 + R) x K columns [k0, k0 + KT) of a row-major FP16 matrix (leading
// dimension ld, rows >= nrows read as zero) into a K-major core-matrix tile.
// Eight consecutive threads fill one core matrix (rows 8g .. 8g + 7, 16 bytes
// each), so a warp writes 512 contiguous bytes of shared memory.
template <int KT>
__device__ __forceinline__ void stage_tile(unsigned char *tile, const __half *src, int64_t ld, int64_t r0, int R,
                                           int64_t nrows, int64_t k0) {
    constexpr int CPR = KT / 8;   // 16-byte chunks per row
    const uint32_t base = su32(tile);
    for (int i = threadIdx.x; i < R * CPR; i += blockDim.x) {
        const int rr = i & 7, c = (i >> 3) % CPR, r = (i / (8 * CPR)) * 8 + rr;
        const uint32_t off = cm<KT>(r, c * 8);
        if (r0 + r < nrows) {
            cp16(base + off, src + (r0 + r) * ld + k0 + c * 8);
        } else {
            *reinterpret_cast<uint4 *>(tile + off) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// Byte offset of element (k, x) of an MN-major core-matrix tile whose MN extent
// is X: core matrices of 8 K-rows x 8 MN-elements (16 contiguous bytes a row),
// MN-adjacent ones 128 B apart, K-adjacent ones X * 16 B apart.  The matrix
// descriptor then takes SBO = 128 (the MN step) and LBO = X * 16 (the K step).
template <int X>
__device__ __forceinline__ uint32_t mn_off(int k, int x) {
    return (uint32_t)((k >> 3) * (X * 16) + (x >> 3) * 128 + (k & 7) * 16 + (x & 7) * 2);
}

// rows [k0, k0 + 128) (the K extent: batch rows) x columns [0, XC) of a
// row-major FP16 matrix (leading dimension ld) into an MN-major tile of MN
// extent X >= XC.  Eight consecutive threads fill one core matrix.
template <int X, int XC>
__device__ __forceinline__ void stage_mn(unsigned char *tile, const __half *src, int64_t ld, int64_t k0) {
    constexpr int XG = XC / 8;    // 16-byte chunks per source row
    const uint32_t base = su32(tile);
    for (int i = threadIdx.x; i < 128 * XG; i += blockDim.x) {
        const int kk = i & 7, xg = (i >> 3) % XG, k = (i / (8 * XG)) * 8 + kk;
        cp16(base + mn_off<X>(k, xg * 8), src + (k0 + k) * ld + xg * 8);
    }
}

enum : int { EPI_FWD = 0, EPI_OUT = 1, EPI_BWD = 2 };

struct TallArgs {
    const __half *A;      // [M][K] row-major (K = KT)
    const __half *Bw;     // [N][K] row-major (the K-major second operand)
    int64_t M;            // batch rows
    int nvalid_cols;      // columns that exist (2P for the output layer)
    const float *bias;    // [N] (EPI_FWD, EPI_OUT)
    float omega0;
    __half *C;            // EPI_FWD: [M][N] cos(omega0 Z) (FP16), kept for the backward pass
    const __half *Cprev;  // EPI_BWD: [M][N] cos(omega0 Z) of the layer below
    const float *T;       // EPI_OUT: [M][ldt] targets
    int ldt;
    __half *O;            // [M][N] FP16 output (H, dY or dZ)
    double *loss;         // EPI_OUT: sum of squared errors (added)
    float *bgrad;         // EPI_OUT: bscale times the column sums of dY (added: the output bias gradient)
    float bscale;
    unsigned int *err;
};

// Column sums over the warp's 32 lanes of v[0 .. CW): lane l ends with the
// sum for column l mod CW in v[0] (a butterfly that halves the live columns at
// each step, CW - 1 shuffles in all).
template <int CW>
__device__ __forceinline__ float warp_colsum(float (&v)[CW], int lane) {
#pragma unroll
    for (int w = CW / 2; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int j = 0; j < w; ++j) {
            const float send = up ? v[j] : v[j + w];
            const float keep = up ? v[j + w] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    float r = v[0];
    if (CW < 32) r += __shfl_xor_sync(0xffffffffu, r, 16);
    return r;
}

// C = A B^T (K = KT, N columns) over all 128-row tiles of A, with the
// epilogue EPI; a persistent kernel with one CTA of 512 threads per SM.  The
// CTA stages B once and takes tiles blockIdx.x, + gridDim.x, ...: two A
// stages and two accumulators in tensor memory, so that while the 16 warps
// run the epilogue of tile i the tensor cores multiply tile i + 1 and tile
// i + 2 loads.  Warp w reads accumulator lanes 32 (w mod 4) .. + 31 (its 32
// rows), columns 32 (w div 4) .. + 31 (all columns for N <= 32, where warps
// 4-15 only stage).  The outputs leave through padded shared memory as whole
// rows.
template <int EPI, int N, int KT>
__global__ void __launch_bounds__(512, 1) tc_tall_kernel(TallArgs g) {
    constexpr int TILE_A = 128 * KT * 2, TILE_B = N * KT * 2;
    constexpr int NA = N < 32 ? 32 : N;   // accumulator columns of one stage
    constexpr int CW = N < 32 ? N : 32;   // columns a warp handles
    extern __shared__ __align__(128) unsigned char tsm[];
    unsigned char *sB = tsm, *sA0 = tsm + TILE_B;
    // [128][N + 8]: O (and C for EPI_FWD) row-major, rows 16-byte aligned and
    // 16 bytes apart in bank order, so that a warp's 16-byte row stores do not
    // collide; the tile then leaves in full 16-byte runs of whole rows
    constexpr int OSTR = N + 8;
    __half *sO = reinterpret_cast<__half *>(tsm + TILE_B + 2 * TILE_A), *sC = sO + 128 * OSTR;
    __shared__ __align__(8) unsigned long long s_mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ double s_loss[16];
    __shared__ float s_cs[4][32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cgrp = warp >> 2;
    const bool epi_warp = (N > 32) || cgrp == 0;
    const int c0 = (N > 32) ? cgrp * 32 : 0;
    const int64_t ntiles = (g.M + 127) / 128;
    const int nt = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    auto tile_row0 = [&](int i) { return (int64_t)(blockIdx.x + (int64_t)i * gridDim.x) * 128; };
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&s_tmem)),
                     "r"(2 * NA)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&s_mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&s_mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (nt > 0) {
        stage_tile<KT>(sB, g.Bw, KT, 0, N, N, 0);
        stage_tile<KT>(sA0, g.A, KT, tile_row0(0), 128, g.M, 0);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (nt > 1) stage_tile<KT>(sA0 + TILE_A, g.A, KT, tile_row0(1), 128, g.M, 0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    auto issue = [&](int i) {   // tile i's MMAs into stage i & 1 (one thread)
        const uint32_t sa = su32(sA0 + (i & 1) * TILE_A), sb = su32(sB);
#pragma unroll
        for (int ks = 0; ks < KT / 16; ++ks)
            mma(tmem + (uint32_t)((i & 1) * NA), sdesc(sa + ks * 256, KT * 16), sdesc(sb + ks * 256, KT * 16),
                idesc(128, N), ks > 0 ? 1u : 0u);
        commit(su32(&s_mbar[i & 1]));
    };
    if (tid == 0 && nt > 0) issue(0);
    bool ok = true;
    double lsum = 0.0;
    float dcol[EPI == EPI_OUT ? CW : 1] = {};   // EPI_OUT: this thread's sums of dY over its rows
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    for (int i = 0; i < nt; ++i) {
        const int b = i & 1;
        ok = __syncthreads_and(mbar_wait(su32(&s_mbar[b]), (i >> 1) & 1));
        if (!ok) break;
        fence_after();
        if (i + 1 < nt) {
            // tile i + 1's operands (the only copies in flight) have landed: multiply
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                fence_after();
                issue(i + 1);
            }
        }
        // stage b is free once tile i's MMAs are done: load tile i + 2 into it
        if (i + 2 < nt) stage_tile<KT>(sA0 + b * TILE_A, g.A, KT, tile_row0(i + 2), 128, g.M, 0);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const int64_t r0 = tile_row0(i), row = r0 + quad * 32 + lane;
        const bool live = row < g.M;
        if (epi_warp) {
            float v[32];
            ld32(tmem + lane_base + (uint32_t)(b * NA + c0), v);
            uint32_t hp[CW / 2], cp[CW / 2];   // FP16 pairs of the output (and of cos for EPI_FWD)
            if constexpr (EPI == EPI_BWD) {
                if (live) {
                    const uint4 *cs = reinterpret_cast<const uint4 *>(g.Cprev + row * N + c0);
#pragma unroll
                    for (int q = 0; q < CW / 8; ++q) {
                        const uint4 u = cs[q];
                        cp[4 * q] = u.x; cp[4 * q + 1] = u.y; cp[4 * q + 2] = u.z; cp[4 * q + 3] = u.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < CW / 2; ++q) cp[q] = 0u;
                }
            }
#pragma unroll
            for (int j = 0; j < CW; j += 2) {
                float o[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int c = c0 + j + e;
                    if constexpr (EPI == EPI_FWD) {
                        float sn, cs;
                        sincos_red(g.omega0 * (v[j + e] + g.bias[c]), &sn, &cs);
                        o[e] = sn;
                        v[j + e] = cs;
                    } else if constexpr (EPI == EPI_OUT) {
                        if (live && c < g.nvalid_cols) {
                            const float d = v[j + e] + g.bias[c] - g.T[row * g.ldt + c];
                            lsum += (double)d * d;
                            o[e] = 2.f * d;
                            dcol[j + e] += o[e];
                        } else {
                            o[e] = 0.f;
                        }
                    } else {
                        const __half2 c2 = *reinterpret_cast<const __half2 *>(&cp[j / 2]);
                        o[e] = v[j + e] * g.omega0 * (e == 0 ? __low2float(c2) : __high2float(c2));
                    }
                }
                const __half2 h2 = __floats2half2_rn(o[0], o[1]);
                hp[j / 2] = *reinterpret_cast<const uint32_t *>(&h2);
                if constexpr (EPI == EPI_FWD) {
                    const __half2 c2 = __floats2half2_rn(v[j], v[j + 1]);
                    cp[j / 2] = *reinterpret_cast<const uint32_t *>(&c2);
                }
            }
            const int rr = quad * 32 + lane;
            {
                uint4 *dst = reinterpret_cast<uint4 *>(sO + rr * OSTR + c0);
#pragma unroll
                for (int q = 0; q < CW / 8; ++q)
                    dst[q] = make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
                if constexpr (EPI == EPI_FWD) {
                    uint4 *cd = reinterpret_cast<uint4 *>(sC + rr * OSTR + c0);
#pragma unroll
                    for (int q = 0; q < CW / 8; ++q)
                        cd[q] = make_uint4(cp[4 * q], cp[4 * q + 1], cp[4 * q + 2], cp[4 * q + 3]);
                }
            }
        }
        fence_before();
        __syncthreads();
        {
            // rows [r0, r0 + 128) of O (and C): N / 8 chunks of 16 bytes per row
            constexpr int RC = N / 8;
            for (int q = tid; q < 128 * RC; q += blockDim.x) {
                const int r = q / RC, j = q - r * RC;
                if (r0 + r < g.M) {
                    *reinterpret_cast<uint4 *>(g.O + (r0 + r) * N + 8 * j) =
                        *reinterpret_cast<const uint4 *>(sO + r * OSTR + 8 * j);
                    if constexpr (EPI == EPI_FWD)
                        *reinterpret_cast<uint4 *>(g.C + (r0 + r) * N + 8 * j) =
                            *reinterpret_cast<const uint4 *>(sC + r * OSTR + 8 * j);
                }
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!ok && tid == 0) atomicExch(g.err, 1u);
    if constexpr (EPI == EPI_OUT) {
        for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) s_loss[warp] = lsum;
        if (cgrp == 0) {
            const float cs = warp_colsum<CW>(dcol, lane);
            if (lane < CW) s_cs[quad][lane] = cs;
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 16; ++w) t += s_loss[w];
            atomicAdd(g.loss, t);
        }
        if (tid < g.nvalid_cols && tid < CW)
            atomicAdd(g.bgrad + tid, g.bscale * (s_cs[0][tid] + s_cs[1][tid] + s_cs[2][tid] + s_cs[3][tid]));
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * NA) : "memory");
    }
}

struct RedArgs {
    const __half *A;      // [K][128] row-major (K the batch): read as an MN-major operand
    const __half *Bw;     // [K][N] row-major: likewise
    int64_t K;            // batch size (multiple of 128)
    float *out;           // += scale C (out[r][c], or out[c][r] when transpose), columns c < ncols
    float *outb;          // BIAS: += scale times the column sums of A (over the batch)
    int ncols, transpose, ldo;
    float scale;
    unsigned int *err;
};

constexpr int RED_STAGES = 3;   // chunks of the batch in flight per CTA (shared-memory stages)

// A split-K slice of C[128][N] = A^T B over the batch (A [K][128], B [K][N]
// row-major, both taken by the tensor cores as MN-major operands, so that
// neither needs a transposed copy), one CTA per SM: the CTA's 128-row chunks
// of the batch stream through RED_STAGES shared-memory stages (two chunks load
// while the tensor cores multiply the third) and accumulate in tensor memory;
// the slice's partial product is then added to the output with 16-byte
// atomic adds.  With BIAS the B tile carries 16 extra columns, the first all
// ones, so accumulator column N holds the column sums of A (the bias gradient
// when A is dZ).
template <int N, bool BIAS>
__global__ void __launch_bounds__(256, 1) tc_red_kernel(RedArgs g) {
    constexpr int KT = 128;
    constexpr int NB = N + (BIAS ? 16 : 0);
    constexpr int TCOLS = NB <= 32 ? 32 : NB <= 64 ? 64 : NB <= 128 ? 128 : 256;
    constexpr int TILE_A = 128 * KT * 2, STAGE = TILE_A + NB * KT * 2;
    static_assert(KT == 128, "chunks of 128 batch rows");
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) unsigned long long s_mbar[RED_STAGES];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t chunks = g.K / KT;
    const int64_t c0 = (int64_t)blockIdx.x * chunks / gridDim.x, c1 = (int64_t)(blockIdx.x + 1) * chunks / gridDim.x;
    const int nk = (int)(c1 - c0);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&s_tmem)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < RED_STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&s_mbar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if constexpr (BIAS) {
        // columns N .. N+15 of every stage's B tile: ones, then zeros (written once)
        for (int i = tid; i < RED_STAGES * 16 * KT; i += blockDim.x) {
            const int s = i / (16 * KT), x = (i / KT) % 16, k = i % KT;
            *reinterpret_cast<__half *>(tsm + s * STAGE + TILE_A + mn_off<NB>(k, N + x)) =
                __float2half(x == 0 ? 1.f : 0.f);
        }
    }
    auto stage = [&](int i) {
        unsigned char *sA = tsm + (i % RED_STAGES) * STAGE;
        const int64_t kc = (c0 + i) * KT;
        stage_mn<128, 128>(sA, g.A, 128, kc);
        stage_mn<NB, N>(sA + TILE_A, g.Bw, N, kc);
    };
    for (int i = 0; i < RED_STAGES - 1; ++i) {
        if (i < nk) stage(i);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    __syncthreads();
    const uint32_t tmem = s_tmem;
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
        const int j = i + RED_STAGES - 1;   // the chunk issued now, into the stage chunk i - 1 used
        if (j < nk) {
            if (i >= 1) {
                bool done = true;
                if (tid == 0) done = mbar_wait(su32(&s_mbar[(i - 1) % RED_STAGES]), ((i - 1) / RED_STAGES) & 1);
                ok = __syncthreads_and(done);
                if (!ok) break;
            }
            stage(j);
        }
        // chunk i's copies are the oldest group but RED_STAGES - 1
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group %0;\n" ::"n"(RED_STAGES - 1) : "memory");
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint32_t sA = su32(tsm + (i % RED_STAGES) * STAGE);
#pragma unroll
            for (int ks = 0; ks < KT / 16; ++ks)   // K slice ks: K-groups 2 ks, 2 ks + 1
                mma(tmem, sdesc2(sA + ks * 2 * (128 * 16), 128 * 16, 128),
                    sdesc2(sA + TILE_A + ks * 2 * (NB * 16), NB * 16, 128), idesc(128, NB, 1, 1),
                    (i > 0 || ks > 0) ? 1u : 0u);
            commit(su32(&s_mbar[i % RED_STAGES]));
        }
    }
    // the last chunk's commit covers every earlier MMA; the earlier phases of
    // its barrier were all waited for above
    if (ok && nk > 0) {
        bool done = true;
        if (tid == 0) done = mbar_wait(su32(&s_mbar[(nk - 1) % RED_STAGES]), ((nk - 1) / RED_STAGES) & 1);
        ok = __syncthreads_and(done);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (!ok && tid == 0) atomicExch(g.err, 1u);
    fence_after();
    // warps w and w + 4 read lanes 32 (w mod 4) .. + 31: half the columns each
    // (all of them for N <= 32), the bias column by the second half
    const int quad = warp & 3, half = warp >> 2, row = quad * 32 + lane;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    constexpr int CW = N < 32 ? N : 32;
    constexpr int NC = N <= 32 ? N : N / 2;
    const bool add = ok && nk > 0;
    if (N > 32 || half == 0) {
        const int cbeg = N > 32 ? half * NC : 0;
#pragma unroll 1
        for (int cc = cbeg; cc < cbeg + NC; cc += 32) {
            float v[32];
            ld32(tmem + lane_base + cc, v);
            if (!add) continue;
            if (g.transpose) {
                // out[c][row]: the warp's 32 rows are contiguous for each column
#pragma unroll
                for (int j = 0; j < CW; ++j)
                    if (cc + j < g.ncols) atomicAdd(g.out + (int64_t)(cc + j) * g.ldo + row, g.scale * v[j]);
            } else {
                float4 *o4 = reinterpret_cast<float4 *>(g.out + (int64_t)row * g.ldo + cc);
#pragma unroll
                for (int j = 0; j < CW; j += 4)
                    if (cc + j + 3 < g.ncols)
                        atomicAdd(o4 + j / 4, make_float4(g.scale * v[j], g.scale * v[j + 1], g.scale * v[j + 2],
                                                          g.scale * v[j + 3]));
            }
        }
    }
    if constexpr (BIAS) {
        if (half == 1) {
            float v[32];
            ld32(tmem + lane_base + N, v);
            if (add) atomicAdd(g.outb + row, g.scale * v[0]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// Layer 1 (5 inputs) forward: Z1 = X W1^T + b1, H1 = sin(omega0 Z1) (FP16) and
// cos(omega0 Z1) (FP16) for the backward pass.  A block takes 128-row tiles
// (blockIdx.x, + gridDim.x, ...): thread (half, r) computes columns 64 half ..
// + 63 of row r; the outputs are staged in padded shared memory and leave as
// whole-row 16-byte stores.
__global__ void __launch_bounds__(256) l1_forward_kernel(const float *X, const float *W1, const float *b1, int64_t B,
                                                         float omega0, __half *C, __half *H) {
    constexpr int STR = TCW + 8;
    extern __shared__ __align__(16) unsigned char l1sm[];
    __half *sH = reinterpret_cast<__half *>(l1sm), *sC = sH + 128 * STR;
    __shared__ float sw[TCW * 5], sb[TCW];
    for (int i = threadIdx.x; i < TCW * 5; i += blockDim.x) sw[i] = W1[i];
    for (int i = threadIdx.x; i < TCW; i += blockDim.x) sb[i] = b1[i];
    __syncthreads();
    const int rr = threadIdx.x & 127, half = threadIdx.x >> 7;
    const int64_t ntiles = (B + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * 128, r = r0 + rr;
        float x[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (r < B)
#pragma unroll
            for (int k = 0; k < 5; ++k) x[k] = X[r * 5 + k];
#pragma unroll 1
        for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 8) {
            uint32_t hp[4], cp[4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                float sn[2], cs[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int o = c0 + j + e;
                    float z = sb[o];
#pragma unroll
                    for (int k = 0; k < 5; ++k) z = fmaf(sw[o * 5 + k], x[k], z);
                    sincos_red(omega0 * z, &sn[e], &cs[e]);
                }
                const __half2 h2 = __floats2half2_rn(sn[0], sn[1]), c2 = __floats2half2_rn(cs[0], cs[1]);
                hp[j / 2] = *reinterpret_cast<const uint32_t *>(&h2);
                cp[j / 2] = *reinterpret_cast<const uint32_t *>(&c2);
            }
            *reinterpret_cast<uint4 *>(sH + rr * STR + c0) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
            *reinterpret_cast<uint4 *>(sC + rr * STR + c0) = make_uint4(cp[0], cp[1], cp[2], cp[3]);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 128 * 16; q += blockDim.x) {
            const int a = q >> 4, j = q & 15;   // row a, chunk j
            if (r0 + a < B) {
                *reinterpret_cast<uint4 *>(H + (r0 + a) * TCW + 8 * j) =
                    *reinterpret_cast<const uint4 *>(sH + a * STR + 8 * j);
                *reinterpret_cast<uint4 *>(C + (r0 + a) * TCW + 8 * j) =
                    *reinterpret_cast<const uint4 *>(sC + a * STR + 8 * j);
            }
        }
        __syncthreads();
    }
}

// Layer 1 gradients: dW1[o][k] += scale sum_r dZ1[r][o] X[r][k] and
// db1[o] += scale sum_r dZ1[r][o].  Thread (g, p) of a block takes outputs
// 2p, 2p + 1 of rows g, g + 4, ... of the block's share, four rows' loads in
// flight at a time; the four row groups meet in shared memory, the blocks in
// atomic adds.
__global__ void __launch_bounds__(256) l1_wgrad_kernel(const __half *dZ, const float *X, int64_t B, float scale,
                                                       float *dW1, float *db1) {
    __shared__ float red[4][TCW][6];
    const int p = threadIdx.x & 63, grp = threadIdx.x >> 6;
    float acc[2][6] = {};
    const int64_t step = (int64_t)gridDim.x * 4;
    int64_t r = (int64_t)blockIdx.x * 4 + grp;
    for (; r + 3 * step < B; r += 4 * step) {
        float2 d[4];
        float x[4][5];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t ru = r + u * step;
            d[u] = __half22float2(*reinterpret_cast<const __half2 *>(dZ + ru * TCW + 2 * p));
#pragma unroll
            for (int k = 0; k < 5; ++k) x[u][k] = X[ru * 5 + k];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                acc[0][k] = fmaf(d[u].x, x[u][k], acc[0][k]);
                acc[1][k] = fmaf(d[u].y, x[u][k], acc[1][k]);
            }
            acc[0][5] += d[u].x;
            acc[1][5] += d[u].y;
        }
    }
    for (; r < B; r += step) {
        const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(dZ + r * TCW + 2 * p));
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float x = X[r * 5 + k];
            acc[0][k] = fmaf(d.x, x, acc[0][k]);
            acc[1][k] = fmaf(d.y, x, acc[1][k]);
        }
        acc[0][5] += d.x;
        acc[1][5] += d.y;
    }
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[grp][2 * p + e][k] = acc[e][k];
    __syncthreads();
    for (int i = threadIdx.x; i < TCW * 6; i += blockDim.x) {
        const int o = i / 6, k = i - o * 6;
        const float t = red[0][o][k] + red[1][o][k] + red[2][o][k] + red[3][o][k];
        atomicAdd(k < 5 ? dW1 + o * 5 + k : db1 + o, scale * t);
    }
}

// FP16 operand copies of up to 8 layers (blockIdx.y): W [rows][cols] (rows >=
// nrow read as zero) and W^T.
struct HalfArgs {
    const float *W[8];
    int nrow[8], rows[8];
    __half *Wh[8], *WhT[8];
    int cols;
};

__global__ void weights_half_kernel(HalfArgs a) {
    const int l = blockIdx.y, rows = a.rows[l], cols = a.cols, nrow = a.nrow[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) {
        const int r = i / cols, c = i - r * cols;
        const __half h = __float2half_rn(r < nrow ? a.W[l][i] : 0.f);
        a.Wh[l][i] = h;
        a.WhT[l][(int64_t)c * rows + r] = h;
    }
}

__global__ void scale_loss_kernel(const double *sum, double inv_b, double *loss_out) { *loss_out += *sum * inv_b; }

}  // namespace

// Work buffers of the tensor-core training path.
struct aw_sur_tc {
    int64_t bcap = 0;
    int nh = 0, nout = 0;              // hidden layers, output columns of the output GEMM (16 or 32)
    std::vector<void *> bufs;
    std::vector<__half *> C;           // [nh][B][128] cos(omega0 Z) of each hidden layer
    std::vector<__half *> H;           // [nh][B][128] activations (FP16)
    __half *dY = nullptr;              // [B][nout] output errors 2 (y - t)
    __half *dZ[2] = {nullptr, nullptr};   // [B][128] gradients at the pre-activations, two layers in flight
    int slices = 0;                    // SMs: CTAs of the persistent and split-K GEMMs
    std::vector<__half *> Wh, WhT;     // layers 2 .. nh+1 (the last: [nout][128] and [128][nout])
    double *lsum = nullptr;
    unsigned int *err = nullptr;
};

int aw_sur_tc_supported(const aw_surrogate *s) {
    return s->cfg.width == TCW && s->cfg.n_hidden >= 2 && (s->cfg.npol == 1 || s->cfg.npol == 4);
}

void aw_sur_tc_free(aw_surrogate *s) {
    if (!s->tc) return;
    for (void *p : s->tc->bufs) aw_dev_free(p);
    delete s->tc;
    s->tc = nullptr;
}

static int tc_alloc(aw_surrogate *s, int64_t B) {
    if (s->tc && s->tc->bcap >= B) return AW_OK;
    aw_sur_tc_free(s);
    aw_sur_tc *t = new aw_sur_tc();
    s->tc = t;
    t->nh = s->cfg.n_hidden;
    t->nout = 2 * s->cfg.npol * s->cfg.npol <= 16 ? 16 : 32;
    auto add = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (aw_dev_malloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        t->bufs.push_back(p);
        return p;
    };
    for (int l = 0; l < t->nh; ++l) {
        t->C.push_back((__half *)add(sizeof(__half) * B * TCW));
        t->H.push_back((__half *)add(sizeof(__half) * B * TCW));
    }
    t->dY = (__half *)add(sizeof(__half) * B * t->nout);
    for (int i = 0; i < 2; ++i) {
        t->dZ[i] = (__half *)add(sizeof(__half) * B * TCW);
    }
    for (int l = 1; l <= t->nh; ++l) {
        const int rows = (l == t->nh) ? t->nout : TCW;
        t->Wh.push_back((__half *)add(sizeof(__half) * rows * TCW));
        t->WhT.push_back((__half *)add(sizeof(__half) * rows * TCW));
    }
    int dev = 0;
    AW_CUDA_TRY(cudaGetDevice(&dev));
    AW_CUDA_TRY(cudaDeviceGetAttribute(&t->slices, cudaDevAttrMultiProcessorCount, dev));
    t->lsum = (double *)add(sizeof(double));
    t->err = (unsigned int *)add(sizeof(unsigned int));
    for (void *p : t->bufs)
        if (!p) return aw_set_error(AW_ENOMEM, "tensor-core training buffers for batch %lld", (long long)B);
    t->bcap = B;
    AW_CUDA_TRY(cudaMemset(t->err, 0, sizeof(unsigned int)));
    return AW_OK;
}

// The FP16 operand copies of layers 2 .. nh+1 from the FP32 master parameters.
int aw_sur_tc_refresh(aw_surrogate *s, cudaStream_t st) {
    aw_sur_tc *t = s->tc;
    if (!t) return AW_OK;
    const int L = (int)s->sizes.size() - 1;
    for (int l0 = 1; l0 < L; l0 += 8) {
        HalfArgs a{};
        a.cols = TCW;
        const int n = std::min(8, L - l0);
        for (int q = 0; q < n; ++q) {
            const int l = l0 + q;
            a.W[q] = s->d_p + s->woff[l];
            a.nrow[q] = s->sizes[l + 1];
            a.rows[q] = (l == L - 1) ? t->nout : TCW;
            a.Wh[q] = t->Wh[l - 1];
            a.WhT[q] = t->WhT[l - 1];
        }
        weights_half_kernel<<<dim3(32, n), 256, 0, st>>>(a);
        AW_CHECK_LAUNCH();
    }
    return AW_OK;
}

template <int EPI, int N, int KT>
static int launch_tall(const TallArgs &g, int sms, cudaStream_t st) {
    constexpr int NA = N < 32 ? 32 : N;
    size_t smem = (size_t)N * KT * 2 + (size_t)2 * 128 * KT * 2 + (size_t)(EPI == EPI_FWD ? 2 : 1) * 128 * (N + 8) * 2;
    // with 256 tensor-memory columns a CTA, more than a third of the SM's shared
    // memory keeps at most two CTAs on an SM, so that their columns fit the 512
    if (2 * NA > 128) smem = std::max<size_t>(smem, 78 * 1024);
    auto kern = tc_tall_kernel<EPI, N, KT>;
    AW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t ntiles = (g.M + 127) / 128;
    kern<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms)), 512, smem, st>>>(g);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

// C[128][N] = A^T B over the batch (A [K][128], B [K][N]) added to out
// (scaled, columns < ncols, optionally transposed; with BIAS the column sums
// of A added to outb): one CTA per SM, each a slice of the batch.
template <int N, bool BIAS>
static int launch_red(const RedArgs &g, int slices, cudaStream_t st) {
    constexpr int NB = N + (BIAS ? 16 : 0);
    // more than half the SM's shared memory: one CTA per SM (tensor memory)
    const size_t smem = std::max<size_t>((size_t)RED_STAGES * (128 + NB) * 128 * 2, 116 * 1024);
    auto kern = tc_red_kernel<N, BIAS>;
    AW_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t chunks = g.K / 128;
    const int nslice = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, slices));
    kern<<<(unsigned)nslice, 256, smem, st>>>(g);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

// Loss (added to *loss_dev, as the mean over the batch) and the gradient of
// the mean loss into s->d_g, for a batch X [B][5], T [B][2P] (B a multiple of
// 128).  The FP16 operand copies must be current (aw_sur_tc_refresh).
int aw_sur_tc_step_grad(aw_surrogate *s, const float *X, const float *T, int B, double *loss_dev, cudaStream_t st) {
    if (!aw_sur_tc_supported(s)) return aw_set_error(AW_EUNSUPPORTED, "tensor-core training needs width 128");
    if (B % 128) return aw_set_error(AW_EINVAL, "tensor-core training batch %d is not a multiple of 128", B);
    const bool fresh = !s->tc || s->tc->bcap < B;
    int rc = tc_alloc(s, B);
    if (rc) return rc;
    if (fresh) {
        rc = aw_sur_tc_refresh(s, st);
        if (rc) return rc;
    }
    aw_sur_tc *t = s->tc;
    const int NH = t->nh, L = NH + 1;           // layers 0 .. NH (the last is the output layer)
    const int NO = 2 * s->cfg.npol * s->cfg.npol;
    const float om = s->cfg.omega0, inv_b = 1.0f / (float)B;
    AW_CUDA_TRY(cudaMemsetAsync(s->d_g, 0, sizeof(float) * s->nparam, st));
    AW_CUDA_TRY(cudaMemsetAsync(t->lsum, 0, sizeof(double), st));
    // ---- forward
    const size_t l1_smem = (size_t)2 * 128 * (TCW + 8) * 2;
    AW_CUDA_TRY(cudaFuncSetAttribute(l1_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l1_smem));
    const unsigned l1_blocks = (unsigned)std::min<int64_t>((B + 127) / 128, 2 * t->slices);
    l1_forward_kernel<<<l1_blocks, 256, l1_smem, st>>>(X, s->d_p + s->woff[0], s->d_p + s->boff[0], B, om, t->C[0],
                                                       t->H[0]);
    AW_CHECK_LAUNCH();
    for (int l = 1; l < NH; ++l) {
        TallArgs g{};
        g.A = t->H[l - 1];
        g.Bw = t->Wh[l - 1];
        g.M = B;
        g.nvalid_cols = TCW;
        g.bias = s->d_p + s->boff[l];
        g.omega0 = om;
        g.C = t->C[l];
        g.O = t->H[l];
        g.err = t->err;
        rc = launch_tall<EPI_FWD, TCW, TCW>(g, t->slices, st);
        if (rc) return rc;
    }
    {
        TallArgs g{};
        g.A = t->H[NH - 1];
        g.Bw = t->Wh[NH - 1];
        g.M = B;
        g.nvalid_cols = NO;
        g.bias = s->d_p + s->boff[L - 1];
        g.T = T;
        g.ldt = NO;
        g.O = t->dY;
        g.loss = t->lsum;
        g.bgrad = s->d_g + s->boff[L - 1];
        g.bscale = inv_b;
        g.err = t->err;
        rc = t->nout == 32 ? launch_tall<EPI_OUT, 32, TCW>(g, t->slices, st)
                           : launch_tall<EPI_OUT, 16, TCW>(g, t->slices, st);
        if (rc) return rc;
    }
    // ---- backward: output layer
    {
        // dW_out^T [128][nout] = H^T dY: rows of the result are the inputs, written transposed
        RedArgs r{};
        r.A = t->H[NH - 1];
        r.Bw = t->dY;
        r.K = B;
        r.out = s->d_g + s->woff[L - 1];
        r.ncols = NO;   // only the first NO columns of the transposed product are parameters
        r.transpose = 1;
        r.ldo = TCW;
        r.scale = inv_b;
        r.err = t->err;
        rc = t->nout == 32 ? launch_red<32, false>(r, t->slices, st) : launch_red<16, false>(r, t->slices, st);
        if (rc) return rc;
        // dH = dY W_out, then dZ of the last hidden layer
        TallArgs g{};
        g.A = t->dY;
        g.Bw = t->WhT[NH - 1];
        g.M = B;
        g.nvalid_cols = TCW;
        g.omega0 = om;
        g.Cprev = t->C[NH - 1];
        g.O = t->dZ[0];
        g.err = t->err;
        rc = t->nout == 32 ? launch_tall<EPI_BWD, TCW, 32>(g, t->slices, st)
                           : launch_tall<EPI_BWD, TCW, 16>(g, t->slices, st);
        if (rc) return rc;
    }
    // ---- backward: hidden layers NH-1 .. 1 (dZ of layer l in buffer cur)
    int cur = 0;
    for (int l = NH - 1; l >= 1; --l) {
        // dW = dZ^T H_prev and db = the column sums of dZ in one GEMM (its rows
        // are added as 16-byte vectors: the offset must be a multiple of 4 floats)
        if (s->woff[l] % 4)
            return aw_set_error(AW_EINVAL, "weight offset %lld not 16-byte aligned", (long long)s->woff[l]);
        RedArgs r{};
        r.A = t->dZ[cur];
        r.Bw = t->H[l - 1];
        r.K = B;
        r.out = s->d_g + s->woff[l];
        r.outb = s->d_g + s->boff[l];
        r.ncols = TCW;
        r.ldo = TCW;
        r.scale = inv_b;
        r.err = t->err;
        rc = launch_red<TCW, true>(r, t->slices, st);
        if (rc) return rc;
        TallArgs g{};
        g.A = t->dZ[cur];
        g.Bw = t->WhT[l - 1];
        g.M = B;
        g.nvalid_cols = TCW;
        g.omega0 = om;
        g.Cprev = t->C[l - 1];
        g.O = t->dZ[cur ^ 1];
        g.err = t->err;
        rc = launch_tall<EPI_BWD, TCW, TCW>(g, t->slices, st);
        if (rc) return rc;
        cur ^= 1;
    }
    // ---- layer 1
    l1_wgrad_kernel<<<2 * t->slices, 256, 0, st>>>(t->dZ[cur], X, B, inv_b, s->d_g + s->woff[0], s->d_g + s->boff[0]);
    AW_CHECK_LAUNCH();
    if (loss_dev) {
        scale_loss_kernel<<<1, 1, 0, st>>>(t->lsum, 1.0 / B, loss_dev);
        AW_CHECK_LAUNCH();
    }
    return AW_OK;
}

// AW_ETIMEOUT if a tensor-core completion wait of the training kernels gave up
// since the last check (synchronises the stream).
int aw_sur_tc_check(aw_surrogate *s, cudaStream_t st) {
    if (!s->tc) return AW_OK;
    unsigned int h = 0;
    AW_CUDA_TRY(cudaMemcpyAsync(&h, s->tc->err, sizeof(h), cudaMemcpyDeviceToHost, st));
    AW_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        cudaMemset(s->tc->err, 0, sizeof(unsigned int));
        return aw_set_error(AW_ETIMEOUT, "a tensor-core completion wait of the surrogate training gave up");
    }
    return AW_OK;
}
