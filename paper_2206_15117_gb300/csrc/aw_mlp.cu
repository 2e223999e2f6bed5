// Learned kernel surrogate: a SIREN-style coordinate MLP that maps kernel
// coordinates (tap offset, w, frequency, parallactic angle) to the P complex
// Mueller kernel values of one tap.  It stands in for the per-bin FFT
// synthesis of arXiv:2206.15117 Sec. 3.2 (kernels are the uv transform of the
// Mueller cells after the anti-aliasing function and the w term) and is
// trained on the tables aw_make_kernels produces.
//
// Definitions (the FP64 oracle states the same ones independently):
//   features x = [d_u/s, d_v/s, 2w/w_max - 1, (f - f_c)/f_h, (chi - chi_c)/chi_h],
//   s = D (S(w)/2 + 1), S(w) the support of the normalisation plane of |w|
//   layers [5, H x n_hidden, 2P]: h = sin(omega0 (W h + b)) for the hidden
//   layers, linear output; flat parameters, per layer W [out][in] then b [out];
//   loss L = (1/B) sum (y - t)^2 with t = kernel / out_scale; Adam with bias
//   correction.  Training and table evaluation run in this file's kernels
//   (FP32 tiled GEMMs, FP32 master weights).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "aw_internal.h"
#include "aw_mlp.h"

namespace {

// ------------------------------------------------------------------ SGEMM
// C(m, n) (+)= sum_k A(m, k) B(k, n), with A(m, k) = A[m*sAm + k*sAk] and
// B(k, n) = B[k*sBk + n*sBn]; C row-major with leading dimension ldc.
// 64 x 64 output tile per CTA, 16-deep K slices staged in shared memory,
// 4 x 4 outputs per thread.  gridDim.z > 1 splits K and adds with atomics.
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float *__restrict__ A, int64_t sAm,
                                                    int64_t sAk, const float *__restrict__ B, int64_t sBk,
                                                    int64_t sBn, float *C, int64_t ldc, int accumulate) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x;
    const int tm = tid / 16, tn = tid % 16;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int kchunk = (K + gridDim.z - 1) / gridDim.z;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    float acc[4][4] = {{0}};
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
        for (int i = tid; i < GK * GT; i += 256) {
            const int kk = i / GT, mm = i % GT;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < kend) ? A[gm * sAm + gk * sAk] : 0.f;
            const int gn = n0 + mm;
            Bs[kk][mm] = (gn < N && gk < kend) ? B[gk * sBk + gn * sBn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tm * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tn * 4 + j;
            if (gn >= N) continue;
            float *c = C + gm * ldc + gn;
            if (gridDim.z > 1 || accumulate) atomicAdd(c, acc[i][j]);
            else *c = acc[i][j];
        }
    }
}

int sgemm(int M, int N, int K, const float *A, int64_t sAm, int64_t sAk, const float *B, int64_t sBk, int64_t sBn,
          float *C, int64_t ldc, int splitk, bool accumulate, cudaStream_t s) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, std::max(1, splitk));
    sgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, accumulate ? 1 : 0);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

// Z += bias (per column); H = sin(omega Z) when `sine`, else H = Z.
__global__ void bias_act_kernel(float *Z, float *H, const float *bias, int64_t rows, int cols, float omega, int sine) {
    const int64_t n = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[i] + bias[i % cols];
        Z[i] = z;
        H[i] = sine ? sinf(omega * z) : z;
    }
}

// dZ = 2 (Y - T) / B and the loss sum
__global__ void loss_grad_kernel(const float *Y, const float *T, float *dZ, int64_t n, float inv_b, double *loss) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dZ[i] = 2.f * d * inv_b;
        s += (double)d * d;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(loss, s * inv_b);
}

// dZ_prev = dH * omega cos(omega Z_prev)
__global__ void sine_back_kernel(const float *dH, const float *Zp, float *dZp, int64_t n, float omega) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dZp[i] = dH[i] * omega * cosf(omega * Zp[i]);
}

// db[c] = sum_r dZ[r][c]
__global__ void colsum_kernel(const float *dZ, int64_t rows, int cols, float *db) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (int64_t r = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.y * blockDim.x)
        s += dZ[r * cols + c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        atomicAdd(&db[c], t);
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// counter-based generator: SplitMix64 (Steele, Lea & Flood, 2014)
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float2 read_k(const void *tab, int storage, int64_t idx) {
    if (storage == AW_STORAGE_FP32) return reinterpret_cast<const float2 *>(tab)[idx];
    if (storage == AW_STORAGE_BF16) return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(tab)[idx]);
    return __half22float2(reinterpret_cast<const __half2 *>(tab)[idx]);
}

struct SetView {
    const void *tab;
    const int64_t *bin_offset;
    const int32_t *bin_support;
    int storage, OS, P, ce, npa, nfb, nw, nbins;
    float inv_scale;
    double w_max;
    const double *pa;     // [npa]
    const double *freq;   // [nfb]
};

struct FeatureScales {
    double D, w_max, f_c, f_h, chi_c, chi_h;
    const int32_t *norm;   // [norm_nw] supports of the normalisation planes
    int norm_nw;
    float out_scale;
};

// The features of a bin that do not depend on the offset: x[2], x[3], x[4]
// and the offset scale dsc (the half support of the normalisation plane of |w|).
struct BinFeat {
    double dsc;
    float x2, x3, x4;
};

__device__ __forceinline__ BinFeat bin_features(const SetView &v, const FeatureScales &fs, int bin) {
    const int p = bin / (v.npa * v.nfb);
    const int a = (bin / v.nfb) % v.npa;
    const int f = bin % v.nfb;
    const double w = v.nw > 1 ? (p + 0.5) * v.w_max / v.nw : 0.0;
    // offsets in units of the half support of the normalisation plane of |w|
    int pn = fs.w_max > 0 ? (int)floor(w * fs.norm_nw / fs.w_max) : 0;
    pn = min(max(pn, 0), fs.norm_nw - 1);
    BinFeat r;
    r.dsc = fs.D * (fs.norm[pn] / 2 + 1);
    r.x2 = (float)(fs.w_max > 0 ? 2.0 * w / fs.w_max - 1.0 : -1.0);
    r.x3 = (float)((v.freq[f] - fs.f_c) / fs.f_h);
    r.x4 = (float)((v.pa[a] - fs.chi_c) / fs.chi_h);
    return r;
}

__device__ __forceinline__ void offset_features(const SetView &v, const BinFeat &bf, int S, int fy, int fx, int jy,
                                                int jx, float *x) {
    const int rho = (S - 2) * v.OS / 2;
    const double du = (double)(jx * v.OS - rho - fx) / v.OS;
    const double dv = (double)(jy * v.OS - rho - fy) / v.OS;
    x[0] = (float)(du / bf.dsc);
    x[1] = (float)(dv / bf.dsc);
    x[2] = bf.x2;
    x[3] = bf.x3;
    x[4] = bf.x4;
}

__device__ __forceinline__ void features_of(const SetView &v, const FeatureScales &fs, int bin, int fy, int fx,
                                            int jy, int jx, float *x) {
    offset_features(v, bin_features(v, fs, bin), v.bin_support[bin], fy, fx, jy, jx, x);
}

// The per-bin features of every bin of a set.
__global__ void bin_features_kernel(SetView v, FeatureScales fs, BinFeat *out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < v.nbins; b += gridDim.x * blockDim.x)
        out[b] = bin_features(v, fs, b);
}

// Random training points from an exact kernel set: bins uniform, then fine
// offset and tap uniform.  A block draws 256 points (one a thread: the draws
// and the features), then gathers their targets together, thread q taking
// element q mod P of point q div P, so that the table reads of one point sit
// side by side and the targets leave as contiguous rows.
__global__ void __launch_bounds__(256) sample_kernel(SetView v, FeatureScales fs, const BinFeat *bf, uint64_t seed,
                                                     int B, float *X, float *T) {
    __shared__ int64_t s_base[256], s_L[256];
    __shared__ int s_tap[256];
    for (int b0 = blockIdx.x * 256; b0 < B; b0 += gridDim.x * 256) {
        const int b = b0 + threadIdx.x;
        if (b < B) {
            const uint64_t r1 = splitmix64(seed ^ ((uint64_t)b * 0x2545F4914F6CDD1Dull));
            const uint64_t r2 = splitmix64(r1);
            const int bin = (int)(r1 % (uint64_t)v.nbins);
            const int S = v.bin_support[bin];
            const uint64_t L = (uint64_t)S * S;
            // pick < OS^2 S^2 <= 2^26 (OS <= 64, S <= 128): the rest in 32-bit arithmetic
            const uint32_t pick = (uint32_t)(r2 % ((uint64_t)v.OS * v.OS * L));
            const int tap = (int)(pick % (uint32_t)L);
            const int off = (int)(pick / (uint32_t)L);
            const int fy = off / v.OS, fx = off % v.OS;
            const int jy = tap / S, jx = tap % S;
            offset_features(v, bf[bin], S, fy, fx, jy, jx, X + (int64_t)b * 5);
            s_base[threadIdx.x] = v.bin_offset[bin] + (int64_t)off * L * v.P;
            s_L[threadIdx.x] = (int64_t)L;
            s_tap[threadIdx.x] = tap;
        }
        __syncthreads();
        const int n = min(256, B - b0);
        for (int q = threadIdx.x; q < n * v.P; q += blockDim.x) {
            const int j = q / v.P, m = q - j * v.P;
            const float2 k = read_k(v.tab, v.storage, s_base[j] + aw_tab_index(v.ce, s_L[j], s_tap[j], m));
            reinterpret_cast<float2 *>(T)[(int64_t)(b0 + j) * v.P + m] =
                make_float2(k.x * v.inv_scale / fs.out_scale, k.y * v.inv_scale / fs.out_scale);
        }
        __syncthreads();
    }
}

// Features of every point of one bin (fy, fx, tap order).
__global__ void bin_points_kernel(SetView v, FeatureScales fs, int bin, int64_t first, int64_t count, float *X) {
    const int S = v.bin_support[bin];
    const int64_t L = (int64_t)S * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = first + i;
        const int tap = (int)(g % L);
        const int off = (int)(g / L);
        features_of(v, fs, bin, off / v.OS, off % v.OS, tap / S, tap % S, X + i * 5);
    }
}

// Store surrogate outputs into a table block (chunked layout, target storage)
// and accumulate the squared error against the exact block.
__global__ void store_points_kernel(SetView exact, FeatureScales fs, int bin, int64_t first, int64_t count,
                                    const float *Y, void *dst, int dst_storage, int dst_ce, float dst_scale,
                                    double *err2, double *ref2) {
    const int S = exact.bin_support[bin];
    const int64_t L = (int64_t)S * S;
    const int P = exact.P;
    double e = 0.0, r = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = first + i;
        const int tap = (int)(g % L);
        const int off = (int)(g / L);
        const int64_t base = exact.bin_offset[bin] + (int64_t)off * L * P;
        for (int m = 0; m < P; ++m) {
            const int64_t o = base + aw_tab_index(exact.ce, L, tap, m);
            const int64_t od = base + aw_tab_index(dst_ce, L, tap, m);
            const float yr = Y[i * 2 * P + 2 * m] * fs.out_scale;
            const float yi = Y[i * 2 * P + 2 * m + 1] * fs.out_scale;
            const float2 k = read_k(exact.tab, exact.storage, o);
            const float kr = k.x * exact.inv_scale, ki = k.y * exact.inv_scale;
            e += (double)(yr - kr) * (yr - kr) + (double)(yi - ki) * (yi - ki);
            r += (double)kr * kr + (double)ki * ki;
            if (dst_storage == AW_STORAGE_FP32)
                reinterpret_cast<float2 *>(dst)[od] = make_float2(yr * dst_scale, yi * dst_scale);
            else if (dst_storage == AW_STORAGE_BF16)
                reinterpret_cast<__nv_bfloat162 *>(dst)[od] = __floats2bfloat162_rn(yr * dst_scale, yi * dst_scale);
            else
                reinterpret_cast<__half2 *>(dst)[od] = __floats2half2_rn(yr * dst_scale, yi * dst_scale);
        }
    }
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(err2, e);
        atomicAdd(ref2, r);
    }
}

int nblk(int64_t n, int t = 256) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

// ------------------------------------------------------------------ surrogate
int aw_sur_alloc_work(aw_surrogate *s, int B) {
    if (B <= s->bcap) return AW_OK;
    for (float *p : s->work) aw_dev_free(p);
    s->work.clear();
    const int L = (int)s->sizes.size() - 1;
    // X, T, Z[l], H[l+1], dZ (max width), dH (max width)
    int maxw = 0;
    for (int w : s->sizes) maxw = std::max(maxw, w);
    auto add = [&](int64_t n) -> float * {
        float *p = nullptr;
        if (aw_dev_malloc(&p, sizeof(float) * std::max<int64_t>(n, 1)) != cudaSuccess) return nullptr;
        s->work.push_back(p);
        return p;
    };
    s->X = add((int64_t)B * s->sizes[0]);
    s->T = add((int64_t)B * s->sizes[L]);
    s->Z.assign(L, nullptr);
    s->H.assign(L + 1, nullptr);
    for (int l = 0; l < L; ++l) {
        s->Z[l] = add((int64_t)B * s->sizes[l + 1]);
        s->H[l + 1] = add((int64_t)B * s->sizes[l + 1]);
    }
    s->dZ = add((int64_t)B * maxw);
    s->dZ2 = add((int64_t)B * maxw);
    s->dH = add((int64_t)B * maxw);
    for (float *p : s->work)
        if (!p) return aw_set_error(AW_ENOMEM, "surrogate work buffers for batch %d", B);
    s->bcap = B;
    return AW_OK;
}

int aw_sur_forward(aw_surrogate *s, const float *X, int B, cudaStream_t st) {
    const int L = (int)s->sizes.size() - 1;
    const float *h = X;
    for (int l = 0; l < L; ++l) {
        const int in = s->sizes[l], out = s->sizes[l + 1];
        const float *W = s->d_p + s->woff[l];
        int rc = sgemm(B, out, in, h, in, 1, W, 1, in, s->Z[l], out, 1, false, st);
        if (rc) return rc;
        bias_act_kernel<<<nblk((int64_t)B * out), 256, 0, st>>>(s->Z[l], s->H[l + 1], s->d_p + s->boff[l], B, out,
                                                                s->cfg.omega0, l < L - 1 ? 1 : 0);
        AW_CHECK_LAUNCH();
        h = s->H[l + 1];
    }
    return AW_OK;
}

// gradient of the loss into s->d_g (zeroed here); *loss_dev receives the loss
int aw_sur_backward(aw_surrogate *s, const float *X, const float *T, int B, double *loss_dev, cudaStream_t st) {
    const int L = (int)s->sizes.size() - 1;
    AW_CUDA_TRY(cudaMemsetAsync(s->d_g, 0, sizeof(float) * s->nparam, st));
    const int nout = s->sizes[L];
    loss_grad_kernel<<<nblk((int64_t)B * nout), 256, 0, st>>>(s->H[L], T, s->dZ, (int64_t)B * nout, 1.0f / B, loss_dev);
    AW_CHECK_LAUNCH();
    float *dz = s->dZ, *dz_other = s->dZ2;
    for (int l = L - 1; l >= 0; --l) {
        const int in = s->sizes[l], out = s->sizes[l + 1];
        const float *hprev = (l == 0) ? X : s->H[l];
        // dW[out][in] = dz^T h_prev   (K = B, split over CTAs)
        const int splitk = std::max(1, std::min(128, B / 512));
        int rc = sgemm(out, in, B, dz, 1, out, hprev, in, 1, s->d_g + s->woff[l], in, splitk, true, st);
        if (rc) return rc;
        dim3 cg(out, std::max(1, std::min(64, B / 1024)));
        colsum_kernel<<<cg, 256, 0, st>>>(dz, B, out, s->d_g + s->boff[l]);
        AW_CHECK_LAUNCH();
        if (l > 0) {
            // dH[B][in] = dz W
            rc = sgemm(B, in, out, dz, out, 1, s->d_p + s->woff[l], in, 1, s->dH, in, 1, false, st);
            if (rc) return rc;
            sine_back_kernel<<<nblk((int64_t)B * in), 256, 0, st>>>(s->dH, s->Z[l - 1], dz_other, (int64_t)B * in,
                                                                    s->cfg.omega0);
            AW_CHECK_LAUNCH();
            std::swap(dz, dz_other);
        }
    }
    return AW_OK;
}

int aw_sur_adam(aw_surrogate *s, float lr, cudaStream_t st) {
    s->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)s->t), c2 = 1.f - std::pow(b2, (float)s->t);
    adam_kernel<<<nblk(s->nparam), 256, 0, st>>>(s->d_p, s->d_g, s->d_m, s->d_v, s->nparam, lr, b1, b2, 1e-8f, c1, c2);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

static SetView view_of(const aw_kernel_set *k, const double *d_pa, const double *d_freq) {
    SetView v;
    v.tab = k->d_table;
    v.bin_offset = k->d_bin_offset;
    v.bin_support = k->d_bin_support;
    v.storage = k->spec.storage;
    v.OS = k->spec.OS;
    v.P = k->P;
    v.ce = k->ce;
    v.npa = k->spec.npa;
    v.nfb = k->spec.nfb;
    v.nw = k->spec.nw;
    v.nbins = k->nbins;
    v.inv_scale = 1.0f / k->scale;
    v.w_max = k->spec.w_max;
    v.pa = d_pa;
    v.freq = d_freq;
    return v;
}

static FeatureScales scales_of(const aw_surrogate *s) {
    FeatureScales f;
    f.D = s->cfg.D;
    f.norm = s->d_norm;
    f.norm_nw = (int)s->norm.size();
    f.w_max = s->cfg.w_max;
    f.f_c = s->cfg.f_c;
    f.f_h = s->cfg.f_h;
    f.chi_c = s->cfg.chi_c;
    f.chi_h = s->cfg.chi_h;
    f.out_scale = s->cfg.out_scale;
    return f;
}

struct DevBins {
    double *pa = nullptr, *freq = nullptr;
    BinFeat *feat = nullptr;   // per-bin features (training)
    ~DevBins() {
        if (pa) aw_dev_free(pa);
        if (freq) aw_dev_free(freq);
        if (feat) aw_dev_free(feat);
    }
};

static int upload_bins(const aw_kernel_set *k, DevBins &d) {
    AW_CUDA_TRY(aw_dev_malloc(&d.pa, sizeof(double) * k->pa.size()));
    AW_CUDA_TRY(aw_dev_malloc(&d.freq, sizeof(double) * k->fbin_freqs.size()));
    AW_CUDA_TRY(cudaMemcpy(d.pa, k->pa.data(), sizeof(double) * k->pa.size(), cudaMemcpyHostToDevice));
    AW_CUDA_TRY(cudaMemcpy(d.freq, k->fbin_freqs.data(), sizeof(double) * k->fbin_freqs.size(), cudaMemcpyHostToDevice));
    return AW_OK;
}

int aw_sur_train(aw_surrogate *s, const aw_kernel_set *k, const aw_train_cfg *tc, aw_train_report *rep,
                 cudaStream_t st) {
    if (k->P * 2 != s->sizes.back())
        return aw_set_error(AW_EINVAL, "surrogate has %d outputs, kernel set needs %d", s->sizes.back(), 2 * k->P);
    const int B = tc->batch;
    int rc = aw_sur_alloc_work(s, B);
    if (rc) return rc;
    DevBins db;
    rc = upload_bins(k, db);
    if (rc) return rc;
    const SetView v = view_of(k, db.pa, db.freq);
    const FeatureScales fs = scales_of(s);
    AW_CUDA_TRY(aw_dev_malloc(&db.feat, sizeof(BinFeat) * v.nbins));
    BinFeat *d_bf = db.feat;
    bin_features_kernel<<<nblk(v.nbins), 256, 0, st>>>(v, fs, d_bf);
    AW_CHECK_LAUNCH();
    double *d_loss = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&d_loss, sizeof(double) * std::max(1, tc->steps)));
    AW_CUDA_TRY(cudaMemsetAsync(d_loss, 0, sizeof(double) * std::max(1, tc->steps), st));
    // the tensor-core path (width 128) takes batches in multiples of 128 rows
    const bool use_tc = aw_sur_use_tc(s) && B % 128 == 0;
    if (use_tc) rc = aw_sur_tc_refresh(s, st);
    const auto t0 = std::chrono::steady_clock::now();
    for (int it = 0; it < tc->steps && rc == AW_OK; ++it) {
        sample_kernel<<<nblk(B), 256, 0, st>>>(v, fs, d_bf, tc->seed + 0x9E3779B97F4A7C15ull * (uint64_t)(it + 1), B,
                                                s->X, s->T);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { rc = aw_set_error(AW_ECUDA, "sample: %s", cudaGetErrorString(e)); break; }
        if (use_tc) {
            rc = aw_sur_tc_step_grad(s, s->X, s->T, B, d_loss + it, st);
        } else {
            rc = aw_sur_forward(s, s->X, B, st);
            if (rc) break;
            rc = aw_sur_backward(s, s->X, s->T, B, d_loss + it, st);
        }
        if (rc) break;
        // cosine decay from lr to lr_final
        const double fr = tc->steps > 1 ? (double)it / (tc->steps - 1) : 1.0;
        const float lr = (float)(tc->lr_final + 0.5 * (tc->lr - tc->lr_final) * (1.0 + std::cos(M_PI * fr)));
        rc = aw_sur_adam(s, lr, st);
        if (rc == AW_OK && use_tc) rc = aw_sur_tc_refresh(s, st);
    }
    if (rc == AW_OK && use_tc) rc = aw_sur_tc_check(s, st);
    std::vector<double> losses(std::max(1, tc->steps));
    if (rc == AW_OK) {
        cudaError_t e = cudaMemcpyAsync(losses.data(), d_loss, sizeof(double) * losses.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = aw_set_error(AW_ECUDA, "train: %s", cudaGetErrorString(e));
    }
    aw_dev_free(d_loss);
    if (rc) return rc;
    const auto t1 = std::chrono::steady_clock::now();
    if (rep) {
        rep->steps = tc->steps;
        rep->loss_first = (float)losses.front();
        // mean of the last 5 % of steps
        const int n = std::max(1, tc->steps / 20);
        double m = 0;
        for (int i = tc->steps - n; i < tc->steps; ++i) m += losses[std::max(0, i)];
        rep->loss_last = (float)(m / n);
        rep->seconds = std::chrono::duration<double>(t1 - t0).count();
    }
    return aw_sur_sync_half(s, st);
}

// Evaluate the surrogate at every table point of `exact`; write the result in
// `out`'s storage; planes whose relative L2 error exceeds `reject_rel` keep
// the exact tables.
int aw_sur_tables(aw_surrogate *s, const aw_kernel_set *exact, aw_kernel_set *out, float reject_rel,
                  float *bin_err_host, cudaStream_t st) {
    const int B = 1 << 16;
    int rc = aw_sur_alloc_work(s, B);
    if (rc) return rc;
    DevBins db;
    rc = upload_bins(exact, db);
    if (rc) return rc;
    const SetView v = view_of(exact, db.pa, db.freq);
    const FeatureScales fs = scales_of(s);
    double *d_err = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&d_err, sizeof(double) * 2 * exact->nbins));
    AW_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(double) * 2 * exact->nbins, st));
    for (int b = 0; b < exact->nbins && rc == AW_OK; ++b) {
        const int S = exact->bin_support[b];
        const int64_t npts = (int64_t)exact->spec.OS * exact->spec.OS * S * S;
        for (int64_t first = 0; first < npts && rc == AW_OK; first += B) {
            const int64_t cnt = std::min<int64_t>(B, npts - first);
            bin_points_kernel<<<nblk(cnt), 256, 0, st>>>(v, fs, b, first, cnt, s->X);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { rc = aw_set_error(AW_ECUDA, "points: %s", cudaGetErrorString(e)); break; }
            rc = aw_sur_forward(s, s->X, (int)cnt, st);
            if (rc) break;
            store_points_kernel<<<nblk(cnt), 256, 0, st>>>(v, fs, b, first, cnt, s->H.back(),
                                                          static_cast<char *>(out->d_table), out->spec.storage,
                                                          out->ce, out->scale, d_err + 2 * b, d_err + 2 * b + 1);
            e = cudaGetLastError();
            if (e != cudaSuccess) { rc = aw_set_error(AW_ECUDA, "store: %s", cudaGetErrorString(e)); break; }
        }
    }
    std::vector<double> err(2 * exact->nbins);
    if (rc == AW_OK) {
        cudaError_t e = cudaMemcpyAsync(err.data(), d_err, sizeof(double) * err.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = aw_set_error(AW_ECUDA, "tables: %s", cudaGetErrorString(e));
    }
    aw_dev_free(d_err);
    if (rc) return rc;
    // per-w-plane rejection: the worst bin of a plane decides for the plane
    const int per = exact->spec.npa * exact->spec.nfb;
    out->n_rejected = 0;
    s->plane_rejected.assign(exact->spec.nw, 0);
    for (int p = 0; p < exact->spec.nw; ++p) {
        double worst = 0;
        for (int j = 0; j < per; ++j) {
            const int b = p * per + j;
            const double rel = err[2 * b + 1] > 0 ? std::sqrt(err[2 * b] / err[2 * b + 1]) : 0.0;
            if (bin_err_host) bin_err_host[b] = (float)rel;
            worst = std::max(worst, rel);
        }
        if (worst > reject_rel) {
            s->plane_rejected[p] = 1;
            for (int j = 0; j < per; ++j) {
                const int b = p * per + j;
                const int S = exact->bin_support[b];
                const int64_t n = (int64_t)exact->spec.OS * exact->spec.OS * S * S * exact->P;
                // exact values into the output storage
                if (exact->spec.storage == out->spec.storage && exact->scale == out->scale) {
                    AW_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(out->d_table) + exact->bin_offset[b] * out->elem_bytes,
                                                static_cast<const char *>(exact->d_table) + exact->bin_offset[b] * exact->elem_bytes,
                                                n * out->elem_bytes, cudaMemcpyDeviceToDevice, st));
                } else {
                    return aw_set_error(AW_EUNSUPPORTED, "fallback needs the same storage for exact and output sets");
                }
            }
            out->n_rejected += per;
        }
    }
    AW_CUDA_TRY(cudaStreamSynchronize(st));
    return AW_OK;
}

__global__ void to_half_kernel(const float *p, __half *h, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = __float2half_rn(p[i]);
}

int aw_sur_sync_half(aw_surrogate *s, cudaStream_t st) {
    to_half_kernel<<<nblk(s->nparam), 256, 0, st>>>(s->d_p, s->d_ph, s->nparam);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

int aw_sur_init(aw_surrogate *s) {
    // the normalisation layout is owned by the surrogate from here on
    s->norm.assign(s->cfg.norm_supports, s->cfg.norm_supports + s->cfg.norm_nw);
    s->cfg.norm_supports = s->norm.data();
    AW_CUDA_TRY(aw_dev_malloc(&s->d_norm, sizeof(int32_t) * s->norm.size()));
    AW_CUDA_TRY(cudaMemcpy(s->d_norm, s->norm.data(), sizeof(int32_t) * s->norm.size(), cudaMemcpyHostToDevice));
    s->sizes.clear();
    s->sizes.push_back(5);
    for (int i = 0; i < s->cfg.n_hidden; ++i) s->sizes.push_back(s->cfg.width);
    s->sizes.push_back(2 * s->cfg.npol * s->cfg.npol);
    const int L = (int)s->sizes.size() - 1;
    s->woff.resize(L);
    s->boff.resize(L);
    int64_t pos = 0;
    for (int l = 0; l < L; ++l) {
        s->woff[l] = pos;
        pos += (int64_t)s->sizes[l + 1] * s->sizes[l];
        s->boff[l] = pos;
        pos += s->sizes[l + 1];
    }
    s->nparam = pos;
    AW_CUDA_TRY(aw_dev_malloc(&s->d_p, sizeof(float) * pos));
    AW_CUDA_TRY(aw_dev_malloc(&s->d_m, sizeof(float) * pos));
    AW_CUDA_TRY(aw_dev_malloc(&s->d_v, sizeof(float) * pos));
    AW_CUDA_TRY(aw_dev_malloc(&s->d_g, sizeof(float) * pos));
    AW_CUDA_TRY(aw_dev_malloc(&s->d_ph, sizeof(__half) * pos));
    // SIREN initialisation (Sitzmann et al. 2020): first layer U(-1/in, 1/in),
    // later layers U(-sqrt(6/in)/omega0, +); biases likewise; host SplitMix64
    std::vector<float> h(pos);
    uint64_t st = s->cfg.seed;
    auto uni = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    for (int l = 0; l < L; ++l) {
        const int in = s->sizes[l], out = s->sizes[l + 1];
        const double lim = (l == 0) ? 1.0 / in : std::sqrt(6.0 / in) / s->cfg.omega0;
        for (int64_t i = 0; i < (int64_t)out * in; ++i) h[s->woff[l] + i] = (float)(lim * uni());
        for (int i = 0; i < out; ++i) h[s->boff[l] + i] = (float)(lim * uni());
    }
    AW_CUDA_TRY(cudaMemcpy(s->d_p, h.data(), sizeof(float) * pos, cudaMemcpyHostToDevice));
    AW_CUDA_TRY(cudaMemset(s->d_m, 0, sizeof(float) * pos));
    AW_CUDA_TRY(cudaMemset(s->d_v, 0, sizeof(float) * pos));
    s->t = 0;
    return aw_sur_sync_half(s, 0);
}

void aw_sur_free(aw_surrogate *s) {
    aw_sur_tc_free(s);
    for (float *p : s->work) aw_dev_free(p);
    if (s->d_rejected) aw_dev_free(s->d_rejected);
    if (s->d_err) aw_dev_free(s->d_err);
    if (s->d_pa) aw_dev_free(s->d_pa);
    if (s->d_norm) aw_dev_free(s->d_norm);
    if (s->d_p) aw_dev_free(s->d_p);
    if (s->d_m) aw_dev_free(s->d_m);
    if (s->d_v) aw_dev_free(s->d_v);
    if (s->d_g) aw_dev_free(s->d_g);
    if (s->d_ph) aw_dev_free(s->d_ph);
}
