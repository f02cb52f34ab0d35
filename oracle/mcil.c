/*
 * ORACLE — test infrastructure only.  Plain, slow FP64 reference for the
 * multi-feature correlation integral (MCIL).  Only tests/, the smoke check
 * and the benchmark's CPU legs may load it.  It shares no code with the
 * CUDA path.  Compiled with -O2 -ffp-contract=off.
 *
 * Paper: arXiv 2203.14742, Sec. 3.1 (multi-feature CIL, Alg. 2): the
 * correlation integral vector of eq. (CIL) is formed for several distances
 * of the pattern difference u = s_i - s_j and the vectors are concatenated;
 * the distances are the L2 norm (eq. norm:L2), the L-infinity norm
 * (eq. norm:Linf), two W^{1,2} norms (eq. norm:W12, the root of the summed
 * squares, and eq. norm:W12prime, the sum of the norms) and two W^{1,inf}
 * norms (eq. norm:W1inf, the maximum, and eq. norm:W1infprime, the sum),
 * with derivatives by finite differences.  Min-max scaled data (Sec. 4,
 * "scaled pattern data"): every species of every pattern mapped to
 * (s - min) / (max - min).
 *
 * Readings of points the paper leaves open:
 *   - a pattern is n_species fields of Gy x Gx nodes (Gy = Gx = G for the
 *     2-D models, Gy = 1 for the 1-D reaction-diffusion-ODE model),
 *     h = 1/(Gx-1);
 *   - derivatives are forward differences of each species field,
 *     Dx s = s[y][x+1] - s[y][x] (Gy x (Gx-1) values) and
 *     Dy s = s[y+1][x] - s[y][x] ((Gy-1) x Gx values, none in 1-D), each
 *     rounded to FP32 once (the derivative patterns are FP32 arrays like
 *     the patterns);
 *   - the derivative of the difference is the difference of the derivative
 *     patterns; discrete norms weight the node sum by h^2 (2-D), so
 *     ||u||_2,h = h ||u||_2, ||Dx u||_2,h = ||Dx s_i - Dx s_j||_2 (the h
 *     of the weight cancels the 1/h of the difference quotient), and
 *     ||Dx u||_inf = (G-1) max |Dx s_i - Dx s_j|;
 *   - the L2 feature itself stays the plain Euclidean norm of the
 *     un-derived patterns (the CIL's own reading: a constant factor only
 *     rescales its radii), so it equals the single-norm CIL exactly;
 *   - with q0, qx, qy the squared distances of the CIL (the exact real sum
 *     of squared differences, rounded once to the nearest double) of the
 *     patterns and of their Dx and Dy patterns, and
 *     m0, mx, my the maxima of |difference| with every difference taken in
 *     FP64 (the same rounded difference as the squared distance uses: exact
 *     unless the two numbers' exponents differ by more than 29), every
 *     feature is one
 *     FP64 expression with each operation rounded:
 *       0 L2        squared value  q0
 *       1 Linf      value          m0
 *       2 W12       squared value  (h^2 q0 + qx) + qy
 *       3 W12'      value          (h sqrt(q0) + sqrt(qx)) + sqrt(qy)
 *       4 W1inf     value          max(m0, max(g mx, g my)),  g = G - 1
 *       5 W1inf'    value          (m0 + g mx) + g my
 *     A "squared" feature is decided like the CIL (R0 = sqrt(max),
 *     d^2 < R_k * R_k); a "value" feature directly (R0 = max, F < R_k);
 *   - min-max scaling: out = fl32(((double)s - min) / (max - min)) in FP64,
 *     0 where max == min;
 *   - in 1-D (Gy = 1) qy = my = 0, and the same expressions are the 1-D
 *     discrete norms up to a constant factor per feature (W12^2 times h,
 *     W12' times sqrt(h)), which leaves the radii's ratios and so the bins
 *     unchanged.
 */
#include <stdint.h>
#include <math.h>

double orc_d2_exact(const float *x, const float *y, int64_t d);

/* Features that are decided on their square (see above). */
int orc_mcil_squared(int feature)
{
    return feature == 0 || feature == 2;
}

/* Min-max scaling of n patterns of n_species fields of `cells` nodes. */
void orc_minmax(const float *X, int64_t n, int64_t cells, int nsp, float *out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int s = 0; s < nsp; ++s) {
            const float *x = X + (i * nsp + s) * cells;
            float *o = out + (i * nsp + s) * cells;
            float mn = x[0], mx = x[0];
            for (int64_t c = 1; c < cells; ++c) {
                if (x[c] < mn) mn = x[c];
                if (x[c] > mx) mx = x[c];
            }
            const double span = (double)mx - (double)mn;
            for (int64_t c = 0; c < cells; ++c) {
                if (mx > mn) {
                    const double num = (double)x[c] - (double)mn;
                    o[c] = (float)(num / span);
                } else {
                    o[c] = 0.0f;
                }
            }
        }
}

/* Forward-difference patterns of Gy x Gx fields: Ax[i][s][y][x] =
   X[i][s][y][x+1] - X[i][s][y][x] (x < Gx-1), Ay[i][s][y][x] =
   X[i][s][y+1][x] - X[i][s][y][x] (y < Gy-1), each the exact difference
   rounded once to FP32. */
void orc_fd(const float *X, int64_t n, int Gy, int Gx, int nsp, float *Ax, float *Ay)
{
    const int64_t cells = (int64_t)Gy * Gx, cex = (int64_t)Gy * (Gx - 1), cey = (int64_t)(Gy - 1) * Gx;
    for (int64_t i = 0; i < n; ++i)
        for (int s = 0; s < nsp; ++s) {
            const float *x = X + (i * nsp + s) * cells;
            float *ax = Ax + (i * nsp + s) * cex;
            float *ay = Ay + (i * nsp + s) * cey;
            for (int y = 0; y < Gy; ++y)
                for (int c = 0; c + 1 < Gx; ++c)
                    ax[(int64_t)y * (Gx - 1) + c] = (float)((double)x[(int64_t)y * Gx + c + 1] -
                                                            (double)x[(int64_t)y * Gx + c]);
            for (int y = 0; y + 1 < Gy; ++y)
                for (int c = 0; c < Gx; ++c)
                    ay[(int64_t)y * Gx + c] = (float)((double)x[(int64_t)(y + 1) * Gx + c] -
                                                      (double)x[(int64_t)y * Gx + c]);
        }
}

/* max_t |x_t - y_t| of two FP32 vectors, each difference in FP64 (rounded
   to nearest; exact unless the exponents differ by more than 29). */
double orc_maxabs(const float *x, const float *y, int64_t d)
{
    double m = 0.0;
    for (int64_t t = 0; t < d; ++t) {
        double a = fabs((double)x[t] - (double)y[t]);
        if (a > m) m = a;
    }
    return m;
}

/* The six feature values of every cross-set pair (features not in `mask`
   are left untouched).  X1, X2: patterns [n][nsp][Gy][Gx]; A*1, A*2 their
   forward-difference patterns (orc_fd).  V[(f * n1 + i) * n2 + j]. */
void orc_mcil_values(const float *X1, const float *Ax1, const float *Ay1, int64_t n1,
                     const float *X2, const float *Ax2, const float *Ay2, int64_t n2,
                     int Gy, int Gx, int nsp, int mask, double *V)
{
    const int64_t d0 = (int64_t)nsp * Gy * Gx;
    const int64_t dex = (int64_t)nsp * Gy * (Gx - 1), dey = (int64_t)nsp * (Gy - 1) * Gx;
    const double g = (double)(Gx - 1);
    const double h = 1.0 / g;
    const double h2 = 1.0 / (g * g);
    const int64_t np = n1 * n2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n1; ++i)
        for (int64_t j = 0; j < n2; ++j) {
            const int64_t q = i * n2 + j;
            const float *x = X1 + i * d0, *y = X2 + j * d0;
            double q0 = 0, qx = 0, qy = 0, m0 = 0, mx = 0, my = 0;
            if (mask & 0x0D) q0 = orc_d2_exact(x, y, d0);
            if (mask & 0x0C) {
                qx = orc_d2_exact(Ax1 + i * dex, Ax2 + j * dex, dex);
                qy = orc_d2_exact(Ay1 + i * dey, Ay2 + j * dey, dey);
            }
            if (mask & 0x32) m0 = orc_maxabs(x, y, d0);
            if (mask & 0x30) {
                mx = orc_maxabs(Ax1 + i * dex, Ax2 + j * dex, dex);
                my = orc_maxabs(Ay1 + i * dey, Ay2 + j * dey, dey);
            }
            if (mask & 0x01) V[0 * np + q] = q0;
            if (mask & 0x02) V[1 * np + q] = m0;
            if (mask & 0x04) {
                double a = h2 * q0;
                a = a + qx;
                a = a + qy;
                V[2 * np + q] = a;
            }
            if (mask & 0x08) {
                double a = h * sqrt(q0);
                a = a + sqrt(qx);
                a = a + sqrt(qy);
                V[3 * np + q] = a;
            }
            if (mask & 0x10) {
                const double bx = g * mx, by = g * my;
                const double b = bx > by ? bx : by;
                V[4 * np + q] = m0 > b ? m0 : b;
            }
            if (mask & 0x20) {
                double a = m0 + g * mx;
                a = a + g * my;
                V[5 * np + q] = a;
            }
        }
}

/* Radii, bins and counts of one feature (Sec. 2.1 with the feature's
   distance): squared features R0 = sqrt(max V), K = #{k : V < R_k * R_k};
   value features R0 = max V, K = #{k : V < R_k}.  law 0: R_k = R_{k-1} / b;
   law 1 (the linear law, Sec. 2.1 / Sec. 3.2): R_min = sqrt(min V) (value
   features: min V), h = (R0 - R_min) / M, R_k = R0 - k h; law 2 (the power
   law with the decay fitted to the range): R_k = R_{k-1} / b with b =
   orc_fitted_b(R0 / R_min, M) (cil.c).
   radii[0] = R0, radii[1..M] = R_1..R_M. */
double orc_fitted_b(double c, int M);
void orc_mcil_bins(const double *V, int64_t np, int squared, int law, double b, int M, double *radii,
                   uint8_t *bins, int64_t *counts)
{
    double mx = 0.0, mn = V[0];
    for (int64_t q = 0; q < np; ++q) {
        if (V[q] > mx) mx = V[q];
        if (V[q] < mn) mn = V[q];
    }
    double R = squared ? sqrt(mx) : mx;
    radii[0] = R;
    if (law == 1) {
        const double Rm = squared ? sqrt(mn) : mn;
        const double h = (R - Rm) / (double)M;
        for (int k = 1; k <= M; ++k) {
            const double kh = (double)k * h;
            radii[k] = R - kh;
        }
    } else {
        if (law == 2) {
            const double Rm = squared ? sqrt(mn) : mn;
            b = orc_fitted_b(R / Rm, M);
        }
        for (int k = 1; k <= M; ++k) {
            R = R / b;
            radii[k] = R;
        }
    }
    for (int k = 0; k < M; ++k) counts[k] = 0;
    for (int64_t q = 0; q < np; ++q) {
        int K = 0;
        for (int k = 1; k <= M; ++k) {
            const double T = squared ? radii[k] * radii[k] : radii[k];
            if (V[q] < T) K = K + 1;
        }
        bins[q] = (uint8_t)K;
        for (int k = 0; k < K; ++k) counts[k] += 1;
    }
}
