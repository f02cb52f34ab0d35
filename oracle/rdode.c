/*
 * ORACLE — test infrastructure only.  Plain, slow FP64 reference for the
 * reaction-diffusion-ODE model.  Only tests/, the smoke check and the
 * benchmark's CPU legs may load it.  It shares no code with the CUDA path.
 * Compiled with -O2 -ffp-contract=off.
 *
 * Paper: arXiv 2203.14742, Sec. 4.3, eq. (rdode): on (0, 1) with zero-flux
 * boundaries, a non-diffusing u coupled to a diffusing w,
 *   u_t = -u - u w + m1 u^2 / (1 + k u^2),
 *   w_t = D w_xx - m3 w - u w + m2 u^2 / (1 + k u^2);
 * Table 1: 64 nodes, t in [0, 50], theta = (m1, m2), D = 1, m3 = 4.1,
 * k = 0.01.  Initial data (Sec. 4.3): u from uniform noise smoothed by
 * repeated moving averages, w = 0.
 *
 * Layout: one realisation is [species 2][N] (u then w), N nodes,
 * h = 1/(N-1).  Parameter vector p[6] = (Du unused, D, m1, m2, m3, k).
 * Discrete operator (the 1-D analogue of App. B.1.1):
 *   Lap(w)_x = ((w_{x+1} + w_{x-1}) - 2 w_x) (N-1)^2, ghost = edge node.
 * Readings (Sec. 4.3 gives neither the noise range nor the smoothing):
 *   - noise: U(lo, hi) per node from the SplitMix64 stream of the group,
 *     output number (r*2)*N + x (the 2-D rule with one row);
 *   - smoothing: n_smooth passes of the 3-node moving average
 *     u_x <- ((u_{x-1} + u_x) + u_{x+1}) / 3 with ghost = edge node (this
 *     keeps the sum of u exactly in real arithmetic), in FP64, then
 *     rounded once to FP32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "sm64.h"

/* Initial state of n_real realisations, out [n_real][2][N] float32. */
void orc_rdode_init(int N, int n_real, double lo, double hi, uint64_t seed, int n_smooth, float *out)
{
    double *a = malloc(sizeof(double) * (size_t)N), *b = malloc(sizeof(double) * (size_t)N);
    for (int r = 0; r < n_real; ++r) {
        for (int x = 0; x < N; ++x) {
            const uint64_t z = orc_sm64_at(seed, (uint64_t)r * 2u * (uint64_t)N + (uint64_t)x);
            const double U = (double)(z >> 11) * 0x1.0p-53;
            const double span = hi - lo;
            a[x] = lo + span * U;
        }
        for (int it = 0; it < n_smooth; ++it) {
            for (int x = 0; x < N; ++x) {
                const double l = x > 0 ? a[x - 1] : a[x];
                const double rr = x < N - 1 ? a[x + 1] : a[x];
                b[x] = ((l + a[x]) + rr) / 3.0;
            }
            memcpy(a, b, sizeof(double) * (size_t)N);
        }
        float *o = out + (int64_t)r * 2 * N;
        for (int x = 0; x < N; ++x) {
            o[x] = (float)a[x];
            o[N + x] = 0.0f;
        }
    }
    free(a);
    free(b);
}

/* F(w) of one realisation, w and F [2][N]. */
void orc_rdode_rhs(int N, const double *p, const double *w, double *F)
{
    const double g2 = (double)(N - 1) * (double)(N - 1);
    const double *u = w, *v = w + N;
    for (int x = 0; x < N; ++x) {
        const double uk = u[x], vk = v[x];
        const double vl = x > 0 ? v[x - 1] : vk, vr = x < N - 1 ? v[x + 1] : vk;
        const double lap = ((vr + vl) - 2.0 * vk) * g2;
        const double uu = uk * uk;
        const double q = uu / (1.0 + p[5] * uu);
        const double uv = uk * vk;
        F[x] = ((-uk) - uv) + p[2] * q;
        F[N + x] = p[1] * lap + (((-(p[4] * vk)) - uv) + p[3] * q);
    }
}

/* Gershgorin bound of the spectral radius of dF/dw at w [2][N]: the u row
   has no diffusion, |f_u| + |f_w|; the w row, with n in-domain neighbours,
   |-n D (N-1)^2 + g_w| + n D (N-1)^2 + |g_u|. */
double orc_rdode_gershgorin(int N, const double *p, const double *w)
{
    const double dd = p[1] * (double)(N - 1) * (double)(N - 1);
    double rho = 0.0;
    for (int x = 0; x < N; ++x) {
        const double u = w[x], v = w[N + x];
        const double den = 1.0 + p[5] * (u * u);
        const double dq = 2.0 * u / (den * den);          /* d/du u^2 / (1 + k u^2) */
        const double fu = (-1.0 - v) + p[2] * dq, fw = -u;
        const double gu = -v + p[3] * dq, gw = -p[4] - u;
        const int n = (x > 0) + (x < N - 1);
        const double ru = fabs(fu) + fabs(fw);
        const double rw = fabs(-(double)n * dd + gw) + (double)n * dd + fabs(gu);
        if (ru > rho) rho = ru;
        if (rw > rho) rho = rw;
    }
    return rho;
}
