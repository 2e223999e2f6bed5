// Kernel synthesis (aw_make_kernels), storage conversion and the PSWF taper.
//
// arXiv:2206.15117 Sec. 3.2: the degridding kernels are the FFT of the cells
// of the Stokes-basis Mueller matrix (Eq. 5) after multiplication by an
// anti-aliasing function and the w-correction term; the gridding kernels come
// from the inverse Mueller matrix.  Sec. 3.3 / Eq. 6: the diagonal beams of a
// copy of M^S are regularised before the inversion.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "aw_internal.h"

// ---------------------------------------------------------------- PSWF (host)
//
// psi_0(x) = sum_k beta_k Pbar_{2k}(x) (Pbar_n = sqrt(n + 1/2) P_n) is the
// eigenvector for the smallest eigenvalue of the prolate operator
// -(1-x^2) d2/dx2 + 2x d/dx + c^2 x^2, a symmetric tridiagonal matrix in the
// even normalised Legendre basis.  Smallest eigenvalue by Sturm-sequence
// bisection, eigenvector by inverse iteration below it (the shifted matrix is
// positive definite, so the tridiagonal solve needs no pivoting).

static int sturm_count_below(const std::vector<double> &d, const std::vector<double> &e, double x) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) cnt++;
    for (size_t i = 1; i < d.size(); ++i) {
        double qq = (q == 0.0) ? 1e-300 : q;
        q = d[i] - x - e[i - 1] * e[i - 1] / qq;
        if (q < 0) cnt++;
    }
    return cnt;
}

aw_pswf aw_pswf_make(double c, int n) {
    std::vector<double> d(n), e(n - 1);
    for (int k = 0; k < n; ++k) {
        const double m = 2.0 * k;
        d[k] = m * (m + 1) + c * c * (2 * m * (m + 1) - 1) / ((2 * m + 3) * (2 * m - 1));
        if (k < n - 1)
            e[k] = c * c * (m + 2) * (m + 1) / ((2 * m + 3) * std::sqrt((2 * m + 1) * (2 * m + 5)));
    }
    double lo = 1e300, hi = -1e300;
    for (int k = 0; k < n; ++k) {
        double r = (k > 0 ? std::fabs(e[k - 1]) : 0.0) + (k < n - 1 ? std::fabs(e[k]) : 0.0);
        lo = std::fmin(lo, d[k] - r);
        hi = std::fmax(hi, d[k] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count_below(d, e, mid) >= 1) hi = mid; else lo = mid;
    }
    const double lam = 0.5 * (lo + hi);
    const double mu = lam - 1e-9 * std::fmax(1.0, std::fabs(lam));
    std::vector<double> x(n, 1.0), cp(n), dp(n);
    for (int it = 0; it < 6; ++it) {
        // Thomas algorithm on (A - mu I) y = x
        double b0 = d[0] - mu;
        cp[0] = (n > 1 ? e[0] : 0.0) / b0;
        dp[0] = x[0] / b0;
        for (int k = 1; k < n; ++k) {
            const double den = (d[k] - mu) - e[k - 1] * cp[k - 1];
            cp[k] = (k < n - 1 ? e[k] : 0.0) / den;
            dp[k] = (x[k] - e[k - 1] * dp[k - 1]) / den;
        }
        std::vector<double> y(n);
        y[n - 1] = dp[n - 1];
        for (int k = n - 2; k >= 0; --k) y[k] = dp[k] - cp[k] * y[k + 1];
        double nrm = 0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (int k = 0; k < n; ++k) x[k] = y[k] / nrm;
    }
    aw_pswf p;
    p.beta = x;
    p.norm = 1.0;
    const double v0 = p.eval(0.0);
    p.norm = 1.0 / v0;  // also fixes the sign: psi(0) = 1
    return p;
}

double aw_pswf::eval(double x) const {
    // Legendre recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}
    double pm1 = 1.0, p = x;  // P_0, P_1
    double acc = beta[0] * std::sqrt(0.5) * pm1;
    const int nmax = 2 * (int)beta.size() - 2;
    for (int m = 1; m < nmax; ++m) {
        const double pn = ((2.0 * m + 1.0) * x * p - m * pm1) / (m + 1.0);
        pm1 = p;
        p = pn;
        const int deg = m + 1;
        if ((deg & 1) == 0) acc += beta[deg / 2] * std::sqrt(deg + 0.5) * p;
    }
    return acc * norm;
}

// ---------------------------------------------------------------- FP64 complex
struct cd {
    double r, i;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.r, -a.i}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.r * s, a.i * s}; }
__device__ __forceinline__ double cabs2(cd a) { return a.r * a.r + a.i * a.i; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    const double den = b.r * b.r + b.i * b.i;
    return {(a.r * b.r + a.i * b.i) / den, (a.i * b.r - a.r * b.i) / den};
}

struct SynthParams {
    int M, MO, S, OS, P, npol, role;
    double F;           // field width, radians
    double w;           // w-plane centre, wavelengths
    double chi;         // parallactic angle
    double lambda;      // wavelength of the beam-frequency bin
    double dish;
    double dxy_r, dxy_i, dyx_r, dyx_i;     // leakage of the first antenna of the baseline
    double dxy2_r, dxy2_i, dyx2_r, dyx2_i; // and of the second
    double eps;
    double point_l, point_m;      // antenna pointing relative to the phase centre
    const double *taper;          // [M], taper[0] = 0
    unsigned long long *bmax;     // [4] max |M^S_pp| as double bits
    cufftDoubleComplex *Z;        // [P][MO][MO]
};

// Correlation -> Stokes (Eq. 4, U read as (XY + YX)/2) and its inverse.
__device__ __forceinline__ cd T_cs(int s, int c) {
    // rows I, Q, U, V; columns XX, XY, YX, YY
    switch (s * 4 + c) {
        case 0: return {0.5, 0};  case 3: return {0.5, 0};
        case 4: return {0.5, 0};  case 7: return {-0.5, 0};
        case 9: return {0.5, 0};  case 10: return {0.5, 0};
        case 13: return {0, -0.5}; case 14: return {0, 0.5};
        default: return {0, 0};
    }
}
__device__ __forceinline__ cd Tinv_cs(int c, int s) {
    // XX = I + Q, XY = U + iV, YX = U - iV, YY = I - Q
    switch (c * 4 + s) {
        case 0: return {1, 0};  case 1: return {1, 0};
        case 6: return {1, 0};  case 7: return {0, 1};
        case 10: return {1, 0}; case 11: return {0, -1};
        case 12: return {1, 0}; case 13: return {-1, 0};
        default: return {0, 0};
    }
}

// Jones matrix E [[1, dxy], [dyx, 1]] R(chi), R = [[c, -s], [s, c]].
__device__ __forceinline__ void jones_at(double E, double sc, double cc, double dxy_r, double dxy_i, double dyx_r,
                                         double dyx_i, cd J[2][2]) {
    J[0][0] = {E * (cc + dxy_r * sc), E * (dxy_i * sc)};
    J[0][1] = {E * (-sc + dxy_r * cc), E * (dxy_i * cc)};
    J[1][0] = {E * (dyx_r * cc + sc), E * (dyx_i * cc)};
    J[1][1] = {E * (-dyx_r * sc + cc), E * (-dyx_i * sc)};
}

// Mueller matrix of a baseline (i, j): M = J_i kron conj(J_j) (Sec. 2.1);
// J_i = J_j for baseline-averaged kernels.
__device__ void mueller_at(const SynthParams &p, double l, double m, cd Mu[16]) {
    // the beam is centred on the pointing
    l -= p.point_l;
    m -= p.point_m;
    const double r = sqrt(l * l + m * m);
    const double x = M_PI * p.dish * r / p.lambda;
    const double E = (x == 0.0) ? 1.0 : 2.0 * j1(x) / x;
    double sc, cc;
    sincos(p.chi, &sc, &cc);
    cd Ji[2][2], Jj[2][2];
    jones_at(E, sc, cc, p.dxy_r, p.dxy_i, p.dyx_r, p.dyx_i, Ji);
    jones_at(E, sc, cc, p.dxy2_r, p.dxy2_i, p.dyx2_r, p.dyx2_i, Jj);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                for (int d = 0; d < 2; ++d)
                    Mu[(2 * a + b) * 4 + (2 * c + d)] = cmul(Ji[a][c], cconj(Jj[b][d]));
}

__device__ void stokes_mueller(const cd Mu[16], cd MS[16]) {
    cd tmp[16];
    for (int a = 0; a < 4; ++a)
        for (int s = 0; s < 4; ++s) {
            cd acc = {0, 0};
            for (int b = 0; b < 4; ++b) acc = cadd(acc, cmul(Mu[a * 4 + b], Tinv_cs(b, s)));
            tmp[a * 4 + s] = acc;
        }
    for (int s = 0; s < 4; ++s)
        for (int t = 0; t < 4; ++t) {
            cd acc = {0, 0};
            for (int a = 0; a < 4; ++a) acc = cadd(acc, cmul(T_cs(s, a), tmp[a * 4 + t]));
            MS[s * 4 + t] = acc;
        }
}

// Gauss-Jordan inverse with partial pivoting, FP64.
__device__ void invert4(const cd A[16], cd out[16]) {
    cd a[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c)
            a[r][c] = (c < 4) ? A[r * 4 + c] : cd{(c - 4 == r) ? 1.0 : 0.0, 0.0};
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        double best = cabs2(a[col][col]);
        for (int r = col + 1; r < 4; ++r) {
            const double v = cabs2(a[r][col]);
            if (v > best) { best = v; piv = r; }
        }
        if (piv != col)
            for (int c = 0; c < 8; ++c) { cd t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        const cd pv = a[col][col];
        for (int c = 0; c < 8; ++c) a[col][c] = cdiv(a[col][c], pv);
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            const cd f = a[r][col];
            for (int c = 0; c < 8; ++c) a[r][c] = csub(a[r][c], cmul(f, a[col][c]));
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out[r * 4 + c] = a[r][c + 4];
}

// Eq. 6: B' = B/|B| (|B| + beta/|B|), beta = ((eps/2) max|B|)^2; |B| clamped
// to 1e-12 max|B| with phase 0 at the null.
__device__ cd regularise(cd B, double bmax, double eps) {
    const double beta = (eps * 0.5 * bmax) * (eps * 0.5 * bmax);
    const double floor_ = 1e-12 * bmax;
    double a = sqrt(cabs2(B));
    cd ph;
    if (a < floor_) { a = floor_; ph = {1.0, 0.0}; }
    else ph = {B.r / a, B.i / a};
    return cscale(ph, a + beta / a);
}

__global__ void synth_bmax_kernel(SynthParams p) {
    const int M = p.M;
    double mx[4] = {0, 0, 0, 0};
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < M * M; idx += gridDim.x * blockDim.x) {
        const int q = idx / M, pp = idx % M;
        const double l = (pp - M / 2) * p.F / M, m = (q - M / 2) * p.F / M;
        cd Mu[16], MS[16];
        mueller_at(p, l, m, Mu);
        stokes_mueller(Mu, MS);
        for (int k = 0; k < 4; ++k) mx[k] = fmax(mx[k], sqrt(cabs2(MS[k * 5])));
    }
    for (int k = 0; k < 4; ++k) {
        double v = mx[k];
        for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(&p.bmax[k], (unsigned long long)__double_as_longlong(v));
    }
}

// Image-domain functions written into the zero-padded FFT buffers.
__global__ void synth_cells_kernel(SynthParams p) {
    const int M = p.M, MO = p.MO;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < M * M; idx += gridDim.x * blockDim.x) {
        const int q = idx / M, pp = idx % M;
        const double tap = p.taper[q] * p.taper[pp];
        if (tap == 0.0) continue;
        const double l = (pp - M / 2) * p.F / M, m = (q - M / 2) * p.F / M;
        const double n = sqrt(1.0 - l * l - m * m);
        double sw, cw;
        sincos(2.0 * M_PI * p.w * (n - 1.0), &sw, &cw);
        const cd wg = {cw * tap, sw * tap};     // psi psi exp(+2 pi i w (n-1))
        const int qq = ((q - M / 2) % MO + MO) % MO;
        const int pc = ((pp - M / 2) % MO + MO) % MO;
        const size_t plane = (size_t)MO * MO;
        const size_t off = (size_t)qq * MO + pc;
        if (p.npol == 1) {
            const cd f = (p.role == AW_ROLE_GRID || p.role == AW_ROLE_BEAM) ? wg : cconj(wg);
            p.Z[off] = make_cuDoubleComplex(f.r, f.i);
            continue;
        }
        cd Mu[16];
        mueller_at(p, l, m, Mu);
        if (p.role == AW_ROLE_DEGRID || p.role == AW_ROLE_BEAM) {
            // degrid: [c][s] = W* (M T^-1)_{c,s}; beam: [s][c] = conj(degrid [c][s])
            const cd wd = cconj(wg);
            for (int c = 0; c < 4; ++c)
                for (int s = 0; s < 4; ++s) {
                    cd acc = {0, 0};
                    for (int b = 0; b < 4; ++b) acc = cadd(acc, cmul(Mu[c * 4 + b], Tinv_cs(b, s)));
                    const cd f = cmul(wd, acc);
                    if (p.role == AW_ROLE_DEGRID)
                        p.Z[(size_t)(c * 4 + s) * plane + off] = make_cuDoubleComplex(f.r, f.i);
                    else
                        p.Z[(size_t)(s * 4 + c) * plane + off] = make_cuDoubleComplex(f.r, -f.i);
                }
            continue;
        }
        cd MS[16], Ginv[16];
        stokes_mueller(Mu, MS);
        for (int k = 0; k < 4; ++k)
            MS[k * 5] = regularise(MS[k * 5], __longlong_as_double((long long)p.bmax[k]), p.eps);
        invert4(MS, Ginv);
        for (int s = 0; s < 4; ++s)
            for (int c = 0; c < 4; ++c) {
                cd acc = {0, 0};
                for (int t = 0; t < 4; ++t) acc = cadd(acc, cmul(Ginv[s * 4 + t], T_cs(t, c)));
                const cd f = cmul(wg, acc);
                if (p.role == AW_ROLE_GRID)
                    p.Z[(size_t)(s * 4 + c) * plane + off] = make_cuDoubleComplex(f.r, f.i);
                else  // adjoint: [c][s] = conj(grid[s][c])
                    p.Z[(size_t)(c * 4 + s) * plane + off] = make_cuDoubleComplex(f.r, -f.i);
            }
    }
}

template <int STORAGE>
__device__ __forceinline__ void store_elem(void *dst, int64_t i, double re, double im);
template <>
__device__ __forceinline__ void store_elem<AW_STORAGE_FP32>(void *dst, int64_t i, double re, double im) {
    reinterpret_cast<float2 *>(dst)[i] = make_float2((float)re, (float)im);
}
template <>
__device__ __forceinline__ void store_elem<AW_STORAGE_BF16>(void *dst, int64_t i, double re, double im) {
    __nv_bfloat162 v;
    v.x = __double2bfloat16(re);
    v.y = __double2bfloat16(im);
    reinterpret_cast<__nv_bfloat162 *>(dst)[i] = v;
}
template <>
__device__ __forceinline__ void store_elem<AW_STORAGE_FP16>(void *dst, int64_t i, double re, double im) {
    __half2 v;
    v.x = __double2half(re);
    v.y = __double2half(im);
    reinterpret_cast<__half2 *>(dst)[i] = v;
}

// Cut S x S taps at OS x OS fine offsets out of the transformed buffers and
// store them in the chunked table layout (aw_tab_index).
template <int STORAGE>
__global__ void synth_extract_kernel(const cufftDoubleComplex *Z, int MO, int S, int OS, int P, int ce,
                                     double scale, void *dst) {
    const int64_t L = (int64_t)S * S;
    const int64_t total = (int64_t)OS * OS * L * P;
    const int rho = (S - 2) * OS / 2;
    const size_t plane = (size_t)MO * MO;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = i;
        const int m = (int)(t % P); t /= P;
        const int jx = (int)(t % S); t /= S;
        const int jy = (int)(t % S); t /= S;
        const int fx = (int)(t % OS); t /= OS;
        const int fy = (int)t;
        const int ky = jy * OS - rho - fy;
        const int kx = jx * OS - rho - fx;
        const int iy = ((ky % MO) + MO) % MO;
        const int ix = ((kx % MO) + MO) % MO;
        const cufftDoubleComplex z = Z[(size_t)m * plane + (size_t)iy * MO + ix];
        const int64_t o = ((int64_t)fy * OS + fx) * L * P + aw_tab_index(ce, L, (int64_t)jy * S + jx, m);
        store_elem<STORAGE>(dst, o, z.x * scale, z.y * scale);
    }
}

// canonical [blocks][L][P] complex64 <-> chunked storage layout
template <int STORAGE>
__global__ void convert_kernel(const float2 *src, void *dst, int64_t n, int L, int P, int ce, float scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % P);
        const int64_t tap = (i / P) % L;
        const int64_t blk = i / ((int64_t)P * L);
        const int64_t o = blk * L * P + aw_tab_index(ce, L, tap, m);
        store_elem<STORAGE>(dst, o, (double)(src[i].x * scale), (double)(src[i].y * scale));
    }
}

template <int STORAGE>
__global__ void export_kernel(const void *src, float2 *dst, int64_t n, int L, int P, int ce, float inv_scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % P);
        const int64_t tap = (i / P) % L;
        const int64_t blk = i / ((int64_t)P * L);
        const int64_t o = blk * L * P + aw_tab_index(ce, L, tap, m);
        float2 v;
        if (STORAGE == AW_STORAGE_FP32) {
            v = reinterpret_cast<const float2 *>(src)[o];
        } else if (STORAGE == AW_STORAGE_BF16) {
            v = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(src)[o]);
        } else {
            v = __half22float2(reinterpret_cast<const __half2 *>(src)[o]);
        }
        dst[i] = make_float2(v.x * inv_scale, v.y * inv_scale);
    }
}

__global__ void absmax_kernel(const float2 *src, int64_t n, unsigned int *out) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fmaxf(fabsf(src[i].x), fabsf(src[i].y)));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

static int blocks_for(int64_t n, int threads, int cap = 65535 * 4) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

int aw_convert_table_scaled(const float2 *src, void *dst, int64_t nblocks, int L, int P, int ce, int storage,
                            float scale, cudaStream_t s) {
    const int64_t n = nblocks * L * P;
    const int nb = blocks_for(n, 256);
    if (storage == AW_STORAGE_FP32) convert_kernel<AW_STORAGE_FP32><<<nb, 256, 0, s>>>(src, dst, n, L, P, ce, scale);
    else if (storage == AW_STORAGE_BF16) convert_kernel<AW_STORAGE_BF16><<<nb, 256, 0, s>>>(src, dst, n, L, P, ce, scale);
    else convert_kernel<AW_STORAGE_FP16><<<nb, 256, 0, s>>>(src, dst, n, L, P, ce, scale);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

int aw_export_table(const void *src, float2 *dst, int64_t nblocks, int L, int P, int ce, int storage,
                    float inv_scale, cudaStream_t s) {
    const int64_t n = nblocks * L * P;
    const int nb = blocks_for(n, 256);
    if (storage == AW_STORAGE_FP32) export_kernel<AW_STORAGE_FP32><<<nb, 256, 0, s>>>(src, dst, n, L, P, ce, inv_scale);
    else if (storage == AW_STORAGE_BF16) export_kernel<AW_STORAGE_BF16><<<nb, 256, 0, s>>>(src, dst, n, L, P, ce, inv_scale);
    else export_kernel<AW_STORAGE_FP16><<<nb, 256, 0, s>>>(src, dst, n, L, P, ce, inv_scale);
    AW_CHECK_LAUNCH();
    return AW_OK;
}

int aw_table_absmax(const float2 *src, int64_t n, float *out_host, cudaStream_t s) {
    unsigned int *d = nullptr;
    AW_CUDA_TRY(aw_dev_malloc(&d, sizeof(unsigned int)));
    cudaMemsetAsync(d, 0, sizeof(unsigned int), s);
    absmax_kernel<<<blocks_for(n, 256, 152 * 16), 256, 0, s>>>(src, n, d);
    unsigned int h = 0;
    cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    aw_dev_free(d);
    if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "absmax: %s", cudaGetErrorString(e));
    unsigned int bits = h;
    float f;
    memcpy(&f, &bits, sizeof(f));
    *out_host = f;
    return AW_OK;
}

static int image_size_for(int S) {
    int M = 16;
    while (M < 2 * S) M *= 2;
    return M;
}

// Validate a spec and fill the geometry of a kernel set (no device work).
int aw_kernel_set_geometry(const aw_kernel_spec *spec, aw_kernel_set *ks) {
    if (!spec) return aw_set_error(AW_EINVAL, "spec is NULL");
    const int N = spec->N;
    if (N < 16 || N > 16384 || (N & (N - 1)))
        return aw_set_error(AW_EINVAL, "N=%d must be a power of two in [16, 16384]", N);
    if (spec->OS < 1 || spec->OS > 64) return aw_set_error(AW_EINVAL, "OS=%d out of [1, 64]", spec->OS);
    if (spec->npol != 1 && spec->npol != 4) return aw_set_error(AW_EINVAL, "npol=%d must be 1 or 4", spec->npol);
    if (spec->nw < 1 || spec->nw > 256) return aw_set_error(AW_EINVAL, "nw=%d out of [1, 256]", spec->nw);
    if (!spec->supports) return aw_set_error(AW_EINVAL, "supports is NULL");
    if (!(spec->dl > 0) || !(spec->W > 0)) return aw_set_error(AW_EINVAL, "dl and W must be positive");
    if (spec->role < 0 || spec->role > 3) return aw_set_error(AW_EINVAL, "bad role %d", spec->role);
    if (!std::isfinite(spec->point_l) || !std::isfinite(spec->point_m) ||
        spec->point_l * spec->point_l + spec->point_m * spec->point_m >= 1.0)
        return aw_set_error(AW_EINVAL, "pointing (%g, %g) not on the visible hemisphere", spec->point_l, spec->point_m);
    if (spec->storage < 0 || spec->storage > 2) return aw_set_error(AW_EINVAL, "bad storage %d", spec->storage);
    const int npa = spec->npa < 1 ? 1 : spec->npa;
    const int nfb = spec->nfb < 1 ? 1 : spec->nfb;
    if (spec->npol == 4 && ((spec->npa >= 1 && !spec->pa) || (spec->nfb >= 1 && !spec->fbin_freqs)))
        return aw_set_error(AW_EINVAL, "pa / fbin_freqs arrays are NULL");
    const int ntype = spec->ntype < 1 ? 1 : spec->ntype;
    if (ntype > 16) return aw_set_error(AW_EINVAL, "ntype=%d out of [0, 16]", spec->ntype);
    if (ntype >= 2 && spec->npol != 4) return aw_set_error(AW_EINVAL, "per-baseline kernels need npol = 4");
    if (ntype >= 2 && !spec->type_leak) return aw_set_error(AW_EINVAL, "type_leak is NULL with ntype=%d", ntype);
    const int nclass = ntype >= 2 ? ntype * ntype : 1;
    if ((int64_t)nclass * spec->nw * npa * nfb > 65535) return aw_set_error(AW_EINVAL, "too many bins");
    ks->ntype = ntype;
    ks->nclass = nclass;
    if (ntype >= 2) {
        ks->type_leak.assign(spec->type_leak, spec->type_leak + 4 * ntype);
        for (double d : ks->type_leak)
            if (!std::isfinite(d)) return aw_set_error(AW_EINVAL, "type_leak holds a non-finite value");
    } else {
        ks->type_leak.clear();
    }
    ks->supports.assign(spec->supports, spec->supports + spec->nw);
    for (int s : ks->supports) {
        if (s < 2 || s > 128) return aw_set_error(AW_EINVAL, "support %d out of [2, 128]", s);
        if (s > N) return aw_set_error(AW_EINVAL, "support %d larger than the grid", s);
        if ((s & 1) && (spec->OS & 1)) return aw_set_error(AW_EINVAL, "odd support %d needs an even OS", s);
    }
    ks->pa.assign(npa, 0.0);
    ks->fbin_freqs.assign(nfb, 1.4e9);
    if (spec->pa) for (int a = 0; a < npa; ++a) ks->pa[a] = spec->pa[a];
    if (spec->fbin_freqs) for (int f = 0; f < nfb; ++f) ks->fbin_freqs[f] = spec->fbin_freqs[f];
    if (spec->npol == 4) {
        for (double f : ks->fbin_freqs)
            if (!(f > 0)) return aw_set_error(AW_EINVAL, "beam frequencies must be positive");
        if (!(spec->dish_d > 0)) return aw_set_error(AW_EINVAL, "dish_d must be positive");
    }
    ks->spec = *spec;
    ks->spec.npa = npa;
    ks->spec.nfb = nfb;
    ks->spec.supports = ks->supports.data();
    ks->spec.pa = ks->pa.data();
    ks->spec.fbin_freqs = ks->fbin_freqs.data();
    ks->spec.ntype = ntype;
    ks->spec.type_leak = ks->type_leak.empty() ? nullptr : ks->type_leak.data();
    ks->P = spec->npol * spec->npol;
    ks->nbins = nclass * spec->nw * npa * nfb;
    ks->bin_support.resize(ks->nbins);
    ks->bin_offset.resize(ks->nbins);
    int64_t pos = 0;
    ks->max_support = 0;
    for (int b = 0; b < ks->nbins; ++b) {
        const int p = (b / (npa * nfb)) % spec->nw;
        const int S = ks->supports[p];
        ks->bin_support[b] = S;
        ks->bin_offset[b] = pos;
        pos += (int64_t)spec->OS * spec->OS * S * S * ks->P;
        if (S > ks->max_support) ks->max_support = S;
    }
    ks->total_elems = pos;
    ks->elem_bytes = spec->storage == AW_STORAGE_FP32 ? 8 : 4;
    ks->ce = std::min(ks->P, 16 / ks->elem_bytes);
    return AW_OK;
}

int aw_kernel_set_alloc(aw_kernel_set *ks) {
    AW_CUDA_TRY(aw_dev_malloc(&ks->d_table, (size_t)ks->total_elems * ks->elem_bytes));
    AW_CUDA_TRY(aw_dev_malloc(&ks->d_bin_support, sizeof(int32_t) * ks->nbins));
    AW_CUDA_TRY(aw_dev_malloc(&ks->d_bin_offset, sizeof(int64_t) * ks->nbins));
    AW_CUDA_TRY(cudaMemcpy(ks->d_bin_support, ks->bin_support.data(), sizeof(int32_t) * ks->nbins,
                           cudaMemcpyHostToDevice));
    AW_CUDA_TRY(cudaMemcpy(ks->d_bin_offset, ks->bin_offset.data(), sizeof(int64_t) * ks->nbins,
                           cudaMemcpyHostToDevice));
    return AW_OK;
}

// Synthesise every bin of `ks` (geometry already filled, tables allocated).
int aw_synthesise(aw_ctx *ctx, aw_kernel_set *ks, cudaStream_t s) {
    const aw_kernel_spec &sp = ks->spec;
    const int npa = sp.npa, nfb = sp.nfb, P = ks->P, OS = sp.OS;
    const double F = sp.N * sp.dl;
    const aw_pswf psw = aw_pswf_make(M_PI * sp.W / 2.0);
    // largest buffer over the planes
    size_t zmax = 0;
    for (int p = 0; p < sp.nw; ++p) {
        const size_t MO = (size_t)image_size_for(ks->supports[p]) * OS;
        zmax = std::max(zmax, (size_t)P * MO * MO);
    }
    cufftDoubleComplex *Z = nullptr;
    double *d_taper = nullptr;
    unsigned long long *d_bmax = nullptr;
    int rc = AW_OK;
    auto cleanup = [&]() {
        if (Z) aw_dev_free(Z);
        if (d_taper) aw_dev_free(d_taper);
        if (d_bmax) aw_dev_free(d_bmax);
    };
    cudaError_t e = aw_dev_malloc(&Z, zmax * sizeof(cufftDoubleComplex));
    if (e == cudaSuccess) e = aw_dev_malloc(&d_taper, 256 * 64 * sizeof(double));
    if (e == cudaSuccess) e = aw_dev_malloc(&d_bmax, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cleanup();
        return aw_set_error(AW_ENOMEM, "synthesis buffers: %s", cudaGetErrorString(e));
    }
    if (sp.storage == AW_STORAGE_FP16) {
        // K(0,0) of the taper-only kernel of the first plane, (sum psi / M)^2,
        // sets a power-of-two scale that lifts the tables into FP16's normal range
        const int M0 = image_size_for(ks->supports[0]);
        double sum = 0;
        for (int i = 1; i < M0; ++i) sum += psw.eval((i - M0 / 2) * 2.0 / M0);
        const double k00 = (sum / M0) * (sum / M0);
        ks->scale = (float)std::ldexp(1.0, (int)std::lround(-std::log2(k00)));
    }
    std::vector<double> taper;
    int lastM = -1;
    for (int p = 0; p < sp.nw && rc == AW_OK; ++p) {
        const int S = ks->supports[p];
        const int M = image_size_for(S);
        const int MO = M * OS;
        if (M != lastM) {
            taper.resize(M);
            for (int i = 0; i < M; ++i) taper[i] = (i == 0) ? 0.0 : psw.eval((i - M / 2) * 2.0 / M);
            e = cudaMemcpyAsync(d_taper, taper.data(), M * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { rc = aw_set_error(AW_ECUDA, "taper upload: %s", cudaGetErrorString(e)); break; }
            lastM = M;
        }
        cufftHandle plan;
        rc = aw_ctx_fft_plan(ctx, 2, MO, P, CUFFT_Z2Z, &plan);
        if (rc != AW_OK) break;
        if (cufftSetStream(plan, s) != CUFFT_SUCCESS) { rc = aw_set_error(AW_ECUDA, "cufftSetStream"); break; }
        const double w = sp.nw > 1 ? (p + 0.5) * sp.w_max / sp.nw : 0.0;
        for (int k = 0; k < ks->nclass && rc == AW_OK; ++k)
        for (int a = 0; a < npa && rc == AW_OK; ++a)
            for (int f = 0; f < nfb && rc == AW_OK; ++f) {
                const int b = ((k * sp.nw + p) * npa + a) * nfb + f;
                SynthParams prm;
                prm.M = M; prm.MO = MO; prm.S = S; prm.OS = OS; prm.P = P; prm.npol = sp.npol;
                prm.role = sp.role; prm.F = F; prm.w = w; prm.chi = ks->pa[a];
                prm.lambda = AW_C_LIGHT / ks->fbin_freqs[f]; prm.dish = sp.dish_d;
                if (ks->nclass > 1) {
                    // class k = ti * ntype + tj: baseline between antennas of types ti and tj
                    const double *li = &ks->type_leak[4 * (k / ks->ntype)];
                    const double *lj = &ks->type_leak[4 * (k % ks->ntype)];
                    prm.dxy_r = li[0]; prm.dxy_i = li[1]; prm.dyx_r = li[2]; prm.dyx_i = li[3];
                    prm.dxy2_r = lj[0]; prm.dxy2_i = lj[1]; prm.dyx2_r = lj[2]; prm.dyx2_i = lj[3];
                } else {
                    prm.dxy_r = sp.d_xy[0]; prm.dxy_i = sp.d_xy[1]; prm.dyx_r = sp.d_yx[0]; prm.dyx_i = sp.d_yx[1];
                    prm.dxy2_r = prm.dxy_r; prm.dxy2_i = prm.dxy_i; prm.dyx2_r = prm.dyx_r; prm.dyx2_i = prm.dyx_i;
                }
                prm.eps = sp.eps; prm.taper = d_taper; prm.bmax = d_bmax; prm.Z = Z;
                prm.point_l = sp.point_l; prm.point_m = sp.point_m;
                const size_t zbytes = (size_t)P * MO * MO * sizeof(cufftDoubleComplex);
                e = cudaMemsetAsync(Z, 0, zbytes, s);
                if (e == cudaSuccess && sp.npol == 4 && (sp.role == AW_ROLE_GRID || sp.role == AW_ROLE_ADJOINT)) {
                    e = cudaMemsetAsync(d_bmax, 0, 4 * sizeof(unsigned long long), s);
                    if (e == cudaSuccess) {
                        synth_bmax_kernel<<<blocks_for((int64_t)M * M, 128, 1024), 128, 0, s>>>(prm);
                        e = cudaGetLastError();
                    }
                }
                if (e == cudaSuccess) {
                    synth_cells_kernel<<<blocks_for((int64_t)M * M, 128, 4096), 128, 0, s>>>(prm);
                    e = cudaGetLastError();
                }
                if (e != cudaSuccess) { rc = aw_set_error(AW_ECUDA, "synthesis kernels: %s", cudaGetErrorString(e)); break; }
                const int dir = (sp.role == AW_ROLE_GRID || sp.role == AW_ROLE_BEAM) ? CUFFT_FORWARD : CUFFT_INVERSE;
                if (cufftExecZ2Z(plan, Z, Z, dir) != CUFFT_SUCCESS) { rc = aw_set_error(AW_ECUDA, "cufftExecZ2Z failed"); break; }
                const double scale = (double)ks->scale / ((double)M * M);
                const int64_t n = (int64_t)OS * OS * S * S * P;
                char *dst = static_cast<char *>(ks->d_table) + ks->bin_offset[b] * ks->elem_bytes;
                const int nb = blocks_for(n, 256);
                if (sp.storage == AW_STORAGE_FP32)
                    synth_extract_kernel<AW_STORAGE_FP32><<<nb, 256, 0, s>>>(Z, MO, S, OS, P, ks->ce, scale, dst);
                else if (sp.storage == AW_STORAGE_BF16)
                    synth_extract_kernel<AW_STORAGE_BF16><<<nb, 256, 0, s>>>(Z, MO, S, OS, P, ks->ce, scale, dst);
                else
                    synth_extract_kernel<AW_STORAGE_FP16><<<nb, 256, 0, s>>>(Z, MO, S, OS, P, ks->ce, scale, dst);
                e = cudaGetLastError();
                if (e != cudaSuccess) { rc = aw_set_error(AW_ECUDA, "extract: %s", cudaGetErrorString(e)); break; }
            }
    }
    e = cudaStreamSynchronize(s);
    if (rc == AW_OK && e != cudaSuccess) rc = aw_set_error(AW_ECUDA, "synthesis: %s", cudaGetErrorString(e));
    cleanup();
    return rc;
}
