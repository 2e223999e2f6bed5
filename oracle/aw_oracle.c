/*
 * FP64 CPU oracle for convolutional AW gridding and degridding.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or table with the CUDA
 * library: every definition here is written out on its own from the method.
 *
 * What it computes (arXiv:2206.15117):
 *   - visibility coordinates in wavelengths (the baseline vector of Eq. 2 is
 *     in units of wavelength), rounded onto the oversampled uv grid;
 *   - gridding: each visibility convolved onto the uv grid with the
 *     oversampled gridding kernel of its (w-plane, parallactic-angle,
 *     frequency) bin (Sec. 3.2: gridding kernels are the uv transform of the
 *     inverse Mueller cells);
 *   - degridding: the gather of a model grid back to visibilities with the
 *     degridding kernels (Sec. 3.2, Eq. 5 cells).
 *
 * Plain loops in input order, no blocking, no reordering.  Build with
 * -ffp-contract=off so that no multiply-add is fused: the coordinate rounding
 * must follow the fixed operation order stated below.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define C_LIGHT 299792458.0

/*
 * Per-visibility coordinate step.
 *
 * For visibility k with row r and channel c:
 *   f  = freq[c] / C_LIGHT                (1/wavelength, one rounding)
 *   u  = uvw[r][0] * f, v = uvw[r][1] * f, w = uvw[r][2] * f
 *   if w < 0: (u, v, w) -> (-u, -v, -w) and flip = 1     (V(-b) = P conj V(b))
 *   xo = u * uscale + half      with uscale = N * dl * OS, half = (N/2) * OS
 *   Xi = floor(xo + 0.5)        (ties go up), same for y
 *   wplane = floor(w * winv) clamped to [0, nw-1], winv = nw / w_max (0: one plane)
 *   bin = (wplane * npa + pa_bin[r]) * nfb + fbin[c]
 *   S  = support[wplane], rho = (S - 2) * OS / 2
 *   x0 = floor((Xi - rho) / OS), fx = Xi - rho - x0 * OS  in [0, OS)
 *   The footprint is cells x0 .. x0 + S - 1: the S cells nearest the
 *   visibility.  Tap j sits at j * OS - rho - fx oversampled units from it.
 *   valid iff x0 >= 0, x0 + S <= N, same for y, and flags[k] == 0
 *
 * Outputs per k: x0, y0, fx, fy, bin, flip, valid.
 */
void oracle_coords(int64_t nvis, const double *uvw, const uint32_t *row_of_vis,
                   const uint16_t *chan_of_vis, const double *freq,
                   const uint8_t *pa_bin, const uint8_t *fbin, const uint8_t *flags,
                   int N, double dl, int OS, int nw, double w_max, int npa, int nfb,
                   const int32_t *support,
                   int32_t *x0_out, int32_t *y0_out, int32_t *fx_out, int32_t *fy_out,
                   int32_t *bin_out, uint8_t *flip_out, uint8_t *valid_out)
{
    const double uscale = (double)N * dl * (double)OS;
    const double half = (double)(N / 2) * (double)OS;
    const double winv = (nw > 1 && w_max > 0.0) ? (double)nw / w_max : 0.0;
    for (int64_t k = 0; k < nvis; ++k) {
        const uint32_t r = row_of_vis[k];
        const uint16_t c = chan_of_vis[k];
        const double f = freq[c] / C_LIGHT;
        double u = uvw[3 * (int64_t)r + 0] * f;
        double v = uvw[3 * (int64_t)r + 1] * f;
        double w = uvw[3 * (int64_t)r + 2] * f;
        uint8_t flip = 0;
        if (w < 0.0) { u = -u; v = -v; w = -w; flip = 1; }
        const double xu = u * uscale;
        const double xv = v * uscale;
        const double xo = xu + half;
        const double yo = xv + half;
        const double xr = xo + 0.5;
        const double yr = yo + 0.5;
        const int64_t Xi = (int64_t)floor(xr);
        const int64_t Yi = (int64_t)floor(yr);
        int wp = 0;
        if (winv > 0.0) {
            const double wt = w * winv;
            wp = (int)floor(wt);
            if (wp < 0) wp = 0;
            if (wp > nw - 1) wp = nw - 1;
        }
        const int pa = pa_bin ? pa_bin[r] : 0;
        const int fb = fbin ? fbin[c] : 0;
        const int bin = (wp * npa + pa) * nfb + fb;
        const int S = support[wp];
        const int64_t rho = (int64_t)(S - 2) * OS / 2;
        const int64_t Ax = Xi - rho, Ay = Yi - rho;
        /* floor division for possibly negative values */
        int64_t ix = Ax / OS; if (Ax < 0 && ix * OS != Ax) ix -= 1;
        int64_t iy = Ay / OS; if (Ay < 0 && iy * OS != Ay) iy -= 1;
        const int64_t ox = Ax - ix * OS;
        const int64_t oy = Ay - iy * OS;
        int valid = 1;
        if (ix < 0 || ix + S > N) valid = 0;
        if (iy < 0 || iy + S > N) valid = 0;
        if (flags && flags[k]) valid = 0;
        x0_out[k] = (int32_t)ix; y0_out[k] = (int32_t)iy;
        fx_out[k] = (int32_t)ox; fy_out[k] = (int32_t)oy;
        bin_out[k] = bin; flip_out[k] = flip; valid_out[k] = (uint8_t)valid;
    }
}

/*
 * Gridding (adjoint of degridding).
 *
 *   G[s][y0+jy][x0+jx] += sum_c K[bin][fy][fx][jy][jx][s*npol+c] * w'_c * V'_c
 *
 * over jy, jx in [0, S).  (V', w') is the visibility after the w<0 flip:
 * npol == 1: V' = conj(V); npol == 4 (XX, XY, YX, YY): V' = P conj(V), where P
 * swaps XY and YX, and the weights are permuted the same way.  A visibility
 * with any non-finite component is skipped and counted.  Kernel tables are
 * complex128, interleaved (re, im); kernel_off[bin] is the element offset of
 * bin's table, a block [OS][OS][S][S][npol*npol].
 *
 * Returns the number of visibilities skipped as non-finite; *wsum receives the
 * sum over gridded visibilities of the mean of their correlation weights.
 */
int64_t oracle_grid(int64_t nvis, int npol, const double *vis, const double *weight,
                    const int32_t *x0, const int32_t *y0, const int32_t *fx,
                    const int32_t *fy, const int32_t *bin, const uint8_t *flip,
                    const uint8_t *valid, const double *ktab, const int64_t *kernel_off,
                    const int32_t *bin_support, int OS, int N, double *grid, double *wsum)
{
    int64_t nonfinite = 0;
    double ws = 0.0;
    const int nm = npol * npol;
    for (int64_t k = 0; k < nvis; ++k) {
        if (!valid[k]) continue;
        double vr[4], vi[4], wt[4];
        int bad = 0;
        for (int c = 0; c < npol; ++c) {
            vr[c] = vis[2 * (k * npol + c) + 0];
            vi[c] = vis[2 * (k * npol + c) + 1];
            wt[c] = weight ? weight[k * npol + c] : 1.0;
            if (!isfinite(vr[c]) || !isfinite(vi[c]) || !isfinite(wt[c])) bad = 1;
        }
        if (bad) { ++nonfinite; continue; }
        if (flip[k]) {
            for (int c = 0; c < npol; ++c) vi[c] = -vi[c];
            if (npol == 4) {
                double t;
                t = vr[1]; vr[1] = vr[2]; vr[2] = t;
                t = vi[1]; vi[1] = vi[2]; vi[2] = t;
                t = wt[1]; wt[1] = wt[2]; wt[2] = t;
            }
        }
        double wmean = 0.0;
        for (int c = 0; c < npol; ++c) wmean += wt[c];
        ws += wmean / (double)npol;
        const int S = bin_support[bin[k]];
        const double *K = ktab + 2 * (kernel_off[bin[k]] +
                                      ((int64_t)fy[k] * OS + fx[k]) * (int64_t)S * S * nm);
        for (int s = 0; s < npol; ++s) {
            double *G = grid + 2 * (int64_t)s * N * N;
            for (int jy = 0; jy < S; ++jy) {
                const int64_t y = y0[k] + jy;
                for (int jx = 0; jx < S; ++jx) {
                    const int64_t x = x0[k] + jx;
                    const double *kt = K + 2 * (((int64_t)jy * S + jx) * nm);
                    double ar = 0.0, ai = 0.0;
                    for (int c = 0; c < npol; ++c) {
                        const double kr = kt[2 * (s * npol + c) + 0];
                        const double ki = kt[2 * (s * npol + c) + 1];
                        const double xr = wt[c] * vr[c];
                        const double xi = wt[c] * vi[c];
                        ar += kr * xr - ki * xi;
                        ai += kr * xi + ki * xr;
                    }
                    G[2 * (y * N + x) + 0] += ar;
                    G[2 * (y * N + x) + 1] += ai;
                }
            }
        }
    }
    *wsum = ws;
    return nonfinite;
}

/*
 * Degridding.
 *
 *   V'_c = sum_s sum_{jy,jx} K[bin][fy][fx][jy][jx][c*npol+s] * G[s][y0+jy][x0+jx]
 *
 * then the w<0 flip is undone: V = conj(V') (npol 1) or P conj(V') (npol 4).
 * Invalid visibilities are written as zero.
 */
void oracle_degrid(int64_t nvis, int npol, const double *grid, const int32_t *x0,
                   const int32_t *y0, const int32_t *fx, const int32_t *fy,
                   const int32_t *bin, const uint8_t *flip, const uint8_t *valid,
                   const double *ktab, const int64_t *kernel_off,
                   const int32_t *bin_support, int OS, int N, double *vis_out)
{
    const int nm = npol * npol;
    for (int64_t k = 0; k < nvis; ++k) {
        double outr[4] = {0, 0, 0, 0}, outi[4] = {0, 0, 0, 0};
        if (valid[k]) {
            const int S = bin_support[bin[k]];
            const double *K = ktab + 2 * (kernel_off[bin[k]] +
                                          ((int64_t)fy[k] * OS + fx[k]) * (int64_t)S * S * nm);
            for (int c = 0; c < npol; ++c) {
                double ar = 0.0, ai = 0.0;
                for (int s = 0; s < npol; ++s) {
                    const double *G = grid + 2 * (int64_t)s * N * N;
                    for (int jy = 0; jy < S; ++jy) {
                        const int64_t y = y0[k] + jy;
                        for (int jx = 0; jx < S; ++jx) {
                            const int64_t x = x0[k] + jx;
                            const double *kt = K + 2 * (((int64_t)jy * S + jx) * nm);
                            const double kr = kt[2 * (c * npol + s) + 0];
                            const double ki = kt[2 * (c * npol + s) + 1];
                            const double gr = G[2 * (y * N + x) + 0];
                            const double gi = G[2 * (y * N + x) + 1];
                            ar += kr * gr - ki * gi;
                            ai += kr * gi + ki * gr;
                        }
                    }
                }
                outr[c] = ar; outi[c] = ai;
            }
            if (flip[k]) {
                for (int c = 0; c < npol; ++c) outi[c] = -outi[c];
                if (npol == 4) {
                    double t;
                    t = outr[1]; outr[1] = outr[2]; outr[2] = t;
                    t = outi[1]; outi[1] = outi[2]; outi[2] = t;
                }
            }
        }
        for (int c = 0; c < npol; ++c) {
            vis_out[2 * (k * npol + c) + 0] = outr[c];
            vis_out[2 * (k * npol + c) + 1] = outi[c];
        }
    }
}

/*
 * Direct evaluation of the measurement equation (Eq. 2) for a set of image
 * pixels, with the sign convention of the degridder (exp(-2 pi i b.s)):
 *
 *   V_k = sum_p I_p exp(-2 pi i (u_k l_p + v_k m_p + w_k (n_p - 1)))
 *
 * u, v, w in wavelengths; l, m direction cosines; n = sqrt(1 - l^2 - m^2).
 * I is complex (interleaved).  Used only on tiny inputs.
 */
void oracle_dft_predict(int64_t nvis, const double *uvw_lambda, int64_t npix,
                        const double *lm, const double *I, double *vis_out)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int64_t k = 0; k < nvis; ++k) {
        const double u = uvw_lambda[3 * k], v = uvw_lambda[3 * k + 1], w = uvw_lambda[3 * k + 2];
        double ar = 0.0, ai = 0.0;
        for (int64_t p = 0; p < npix; ++p) {
            const double l = lm[2 * p], m = lm[2 * p + 1];
            const double n = sqrt(1.0 - l * l - m * m);
            const double ph = -twopi * (u * l + v * m + w * (n - 1.0));
            const double c = cos(ph), s = sin(ph);
            const double ir = I[2 * p], ii = I[2 * p + 1];
            ar += ir * c - ii * s;
            ai += ir * s + ii * c;
        }
        vis_out[2 * k] = ar;
        vis_out[2 * k + 1] = ai;
    }
}

/*
 * Adjoint of oracle_dft_predict (the direct "dirty image"):
 *
 *   D_p = sum_k V_k exp(+2 pi i (u_k l_p + v_k m_p + w_k (n_p - 1)))
 */
void oracle_dft_adjoint(int64_t nvis, const double *uvw_lambda, const double *vis,
                        int64_t npix, const double *lm, double *img_out)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int64_t p = 0; p < npix; ++p) {
        const double l = lm[2 * p], m = lm[2 * p + 1];
        const double n = sqrt(1.0 - l * l - m * m);
        double ar = 0.0, ai = 0.0;
        for (int64_t k = 0; k < nvis; ++k) {
            const double u = uvw_lambda[3 * k], v = uvw_lambda[3 * k + 1], w = uvw_lambda[3 * k + 2];
            const double ph = twopi * (u * l + v * m + w * (n - 1.0));
            const double c = cos(ph), s = sin(ph);
            const double vr = vis[2 * k], vi = vis[2 * k + 1];
            ar += vr * c - vi * s;
            ai += vr * s + vi * c;
        }
        img_out[2 * p] = ar;
        img_out[2 * p + 1] = ai;
    }
}
