/*
 * FP64 reference loops for separable W-projection gridding and degridding.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct CPU
 * oracle that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never does.  It shares no code with the CUDA sources.
 *
 * Conventions (stated once, used by every function below):
 *   - complex numbers are interleaved (re, im) doubles;
 *   - the grid is N x N, row-major [v-cell][u-cell];
 *   - a visibility located at cell (cu, cv) with oversample indices (ou, ov)
 *     and plane p touches the S x S cells (cv - S/2 + 1 + k, cu - S/2 + 1 + j),
 *     j, k = 0..S-1;
 *   - taps[p][o][j] (complex) is the 1-D kernel value for footprint column j
 *     at oversample offset o of plane p; the separable functions take the
 *     v-direction values from taps_v when it is not NULL (the facet screens
 *     of Sec. 4.1 differ between l and m), else from taps;
 *   - conj[i] != 0 means w_i < 0: the kernel used is the complex conjugate of
 *     the |w| plane's kernel;
 *   - keep[i] == 0 means the visibility was dropped (footprint off the grid or
 *     |w| beyond the last plane) and is skipped;
 *   - wrap != 0 makes cell indices periodic modulo N (used only to pin the
 *     method against its continuous definition with full support).
 * Sums run over visibilities in input order, in plain double arithmetic.
 */
#include <stdint.h>
#include <stddef.h>

static int64_t wrap_index(int64_t x, int32_t N)
{
    int64_t r = x % N;
    return r < 0 ? r + N : r;
}

/*
 * Separable gridder, Sec. 5: the update of cell (u, v) by visibility i is
 * W_i V_i F1(u - u_i) F1(v - v_i); the partial product W_i V_i F1(u - u_i) is
 * formed once per footprint column and reused down every row.
 */
void oracle_grid_separable(int64_t nvis, int32_t N, int32_t S, int32_t OS,
                           const int32_t *cu, const int32_t *cv,
                           const int32_t *ou, const int32_t *ov,
                           const int32_t *plane, const uint8_t *conj,
                           const uint8_t *keep, const double *vis,
                           const double *weight, const double *taps,
                           const double *taps_v, int32_t wrap, double *grid)
{
    double pu_re[1024], pu_im[1024];
    for (int64_t i = 0; i < nvis; ++i) {
        if (!keep[i])
            continue;
        double wgt = weight ? weight[i] : 1.0;
        double vr = wgt * vis[2 * i], vi = wgt * vis[2 * i + 1];
        double sgn = conj[i] ? -1.0 : 1.0;
        const double *tu = taps + 2 * (((int64_t)plane[i] * OS + ou[i]) * S);
        const double *tv = (taps_v ? taps_v : taps) + 2 * (((int64_t)plane[i] * OS + ov[i]) * S);
        for (int j = 0; j < S; ++j) {
            double tr = tu[2 * j], ti = sgn * tu[2 * j + 1];
            pu_re[j] = vr * tr - vi * ti;
            pu_im[j] = vr * ti + vi * tr;
        }
        for (int k = 0; k < S; ++k) {
            double sr = tv[2 * k], si = sgn * tv[2 * k + 1];
            int64_t y = (int64_t)cv[i] - S / 2 + 1 + k;
            if (wrap)
                y = wrap_index(y, N);
            for (int j = 0; j < S; ++j) {
                int64_t x = (int64_t)cu[i] - S / 2 + 1 + j;
                if (wrap)
                    x = wrap_index(x, N);
                double *g = grid + 2 * (y * N + x);
                g[0] += pu_re[j] * sr - pu_im[j] * si;
                g[1] += pu_re[j] * si + pu_im[j] * sr;
            }
        }
    }
}

/*
 * Separable degridder (prediction, Sec. 2; its use for prediction is noted in
 * Sec. 6): V_i = W_i * sum_k conj(tv[k]) * sum_j conj(tu[j]) * X[y_k][x_j],
 * the exact adjoint of oracle_grid_separable.  Dropped visibilities get 0.
 */
void oracle_degrid_separable(int64_t nvis, int32_t N, int32_t S, int32_t OS,
                             const int32_t *cu, const int32_t *cv,
                             const int32_t *ou, const int32_t *ov,
                             const int32_t *plane, const uint8_t *conj,
                             const uint8_t *keep, const double *grid,
                             const double *weight, const double *taps,
                             const double *taps_v, int32_t wrap, double *vis_out)
{
    for (int64_t i = 0; i < nvis; ++i) {
        vis_out[2 * i] = 0.0;
        vis_out[2 * i + 1] = 0.0;
        if (!keep[i])
            continue;
        double sgn = conj[i] ? -1.0 : 1.0;
        const double *tu = taps + 2 * (((int64_t)plane[i] * OS + ou[i]) * S);
        const double *tv = (taps_v ? taps_v : taps) + 2 * (((int64_t)plane[i] * OS + ov[i]) * S);
        double acc_re = 0.0, acc_im = 0.0;
        for (int k = 0; k < S; ++k) {
            int64_t y = (int64_t)cv[i] - S / 2 + 1 + k;
            if (wrap)
                y = wrap_index(y, N);
            double row_re = 0.0, row_im = 0.0;
            for (int j = 0; j < S; ++j) {
                int64_t x = (int64_t)cu[i] - S / 2 + 1 + j;
                if (wrap)
                    x = wrap_index(x, N);
                /* conj of the kernel actually used for gridding */
                double tr = tu[2 * j], ti = -sgn * tu[2 * j + 1];
                const double *g = grid + 2 * (y * N + x);
                row_re += tr * g[0] - ti * g[1];
                row_im += tr * g[1] + ti * g[0];
            }
            double sr = tv[2 * k], si = -sgn * tv[2 * k + 1];
            acc_re += sr * row_re - si * row_im;
            acc_im += sr * row_im + si * row_re;
        }
        double wgt = weight ? weight[i] : 1.0;
        vis_out[2 * i] = wgt * acc_re;
        vis_out[2 * i + 1] = wgt * acc_im;
    }
}

/*
 * Exact (non-separable) W-projection gridder, Sec. 2: the full 2-D kernel
 * table2d[p][ov][ou][k][j] = F_w(j - S/2 + 1 - ou/OS, k - S/2 + 1 - ov/OS)
 * is looked up per cell.  This is the 3-D lookup table the paper replaces.
 */
void oracle_grid_exact2d(int64_t nvis, int32_t N, int32_t S, int32_t OS,
                         const int32_t *cu, const int32_t *cv,
                         const int32_t *ou, const int32_t *ov,
                         const int32_t *plane, const uint8_t *conj,
                         const uint8_t *keep, const double *vis,
                         const double *weight, const double *table2d,
                         int32_t wrap, double *grid)
{
    for (int64_t i = 0; i < nvis; ++i) {
        if (!keep[i])
            continue;
        double wgt = weight ? weight[i] : 1.0;
        double vr = wgt * vis[2 * i], vi = wgt * vis[2 * i + 1];
        double sgn = conj[i] ? -1.0 : 1.0;
        const double *K = table2d +
            2 * ((((int64_t)plane[i] * OS + ov[i]) * OS + ou[i]) * S * S);
        for (int k = 0; k < S; ++k) {
            int64_t y = (int64_t)cv[i] - S / 2 + 1 + k;
            if (wrap)
                y = wrap_index(y, N);
            for (int j = 0; j < S; ++j) {
                int64_t x = (int64_t)cu[i] - S / 2 + 1 + j;
                if (wrap)
                    x = wrap_index(x, N);
                double kr = K[2 * (k * S + j)], ki = sgn * K[2 * (k * S + j) + 1];
                double *g = grid + 2 * (y * N + x);
                g[0] += vr * kr - vi * ki;
                g[1] += vr * ki + vi * kr;
            }
        }
    }
}

/*
 * Correction pass with the stored correction F_w - F~_w (Sec. 7: the exact
 * kernel minus the separable one, kept in a full 2-D table).  The table holds
 * Sr x Sr values for the central footprint cells (first one at column / row
 * k0 = (S - Sr) / 2 of the S x S footprint) at OSr oversample offsets per
 * axis: fine offset o uses the coarse entry o / (OS / OSr).  Layout
 * res[plane][ov][ou][k][j].  Gridding adds W V R (conj(R) for w < 0);
 * degridding is its exact adjoint and ADDS W sum conj(kernel) X to vis_out.
 */
void oracle_grid_residual(int64_t nvis, int32_t N, int32_t S, int32_t OS, int32_t Sr,
                          int32_t OSr, const int32_t *cu, const int32_t *cv,
                          const int32_t *ou, const int32_t *ov, const int32_t *plane,
                          const uint8_t *conj, const uint8_t *keep, const double *vis,
                          const double *weight, const double *res, double *grid)
{
    const int32_t step = OS / OSr, k0 = (S - Sr) / 2;
    for (int64_t i = 0; i < nvis; ++i) {
        if (!keep[i])
            continue;
        double wgt = weight ? weight[i] : 1.0;
        double vr = wgt * vis[2 * i], vi = wgt * vis[2 * i + 1];
        double sgn = conj[i] ? -1.0 : 1.0;
        const double *R = res + 2 * ((((int64_t)plane[i] * OSr + ov[i] / step) * OSr +
                                      ou[i] / step) * Sr * Sr);
        for (int k = 0; k < Sr; ++k) {
            int64_t y = (int64_t)cv[i] - S / 2 + 1 + k0 + k;
            for (int j = 0; j < Sr; ++j) {
                int64_t x = (int64_t)cu[i] - S / 2 + 1 + k0 + j;
                double rr = R[2 * (k * Sr + j)], ri = sgn * R[2 * (k * Sr + j) + 1];
                double *g = grid + 2 * (y * N + x);
                g[0] += vr * rr - vi * ri;
                g[1] += vr * ri + vi * rr;
            }
        }
    }
}

void oracle_degrid_residual(int64_t nvis, int32_t N, int32_t S, int32_t OS, int32_t Sr,
                            int32_t OSr, const int32_t *cu, const int32_t *cv,
                            const int32_t *ou, const int32_t *ov, const int32_t *plane,
                            const uint8_t *conj, const uint8_t *keep, const double *grid,
                            const double *weight, const double *res, double *vis_out)
{
    const int32_t step = OS / OSr, k0 = (S - Sr) / 2;
    for (int64_t i = 0; i < nvis; ++i) {
        if (!keep[i])
            continue;
        double sgn = conj[i] ? -1.0 : 1.0;
        const double *R = res + 2 * ((((int64_t)plane[i] * OSr + ov[i] / step) * OSr +
                                      ou[i] / step) * Sr * Sr);
        double ar = 0.0, ai = 0.0;
        for (int k = 0; k < Sr; ++k) {
            int64_t y = (int64_t)cv[i] - S / 2 + 1 + k0 + k;
            for (int j = 0; j < Sr; ++j) {
                int64_t x = (int64_t)cu[i] - S / 2 + 1 + k0 + j;
                /* conj of the kernel used for gridding */
                double rr = R[2 * (k * Sr + j)], ri = -sgn * R[2 * (k * Sr + j) + 1];
                const double *g = grid + 2 * (y * N + x);
                ar += rr * g[0] - ri * g[1];
                ai += rr * g[1] + ri * g[0];
            }
        }
        double wgt = weight ? weight[i] : 1.0;
        vis_out[2 * i] += wgt * ar;
        vis_out[2 * i + 1] += wgt * ai;
    }
}
