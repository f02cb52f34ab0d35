/*
 * ORACLE — test infrastructure only.  Plain, slow FP64 reference for the
 * reaction-diffusion part of the CIL hot path.  Only tests/, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.  It shares no code with the CUDA path.
 *
 * Compiled with -O2 -ffp-contract=off, so every a*b+c below is two roundings.
 *
 * Paper: arXiv 2203.14742.
 *   Reaction-diffusion system, eq. (rdgen), Sec. 4.1; kinetics FHN eq.
 *   (introduction:0) and GM eq. (gmSystem); homogeneous equilibria, Sec. 4.1;
 *   initial state = equilibrium + uniform noise, Sec. 4.1; method of lines,
 *   5-point Laplacian and mirrored Neumann ghosts, App. B.1.1; explicit Euler,
 *   Sec. 5.1.
 *
 * Species order is (u, v).  Mapping onto the paper's (v, w) notation:
 *   FHN:  u = w (membrane potential), v = v (recovery), mu = 1,
 *         Du = nu_2, Dv = nu_1, eps, a = alpha.
 *         F_u = Du*Lap(u) + u - u^3 - v,  F_v = Dv*Lap(v) + eps*(u - a*v).
 *   GM:   u = v (activator), v = w (inhibitor), mu_w = 1, mu = mu_v, with an
 *         overall rate rho.
 *         F_u = Du*Lap(u) + rho*(u^2/v - mu*u),  F_v = Dv*Lap(v) + rho*(u^2 - v).
 *   DIFF: pure diffusion (reaction switched off), a degenerate case used to
 *         pin the discrete Laplacian.
 *   BZ:   the Brusselator ("BZ" in the paper's Table 1), u = v, v = w,
 *         Du = nu_1, Dv = nu_2:
 *         F_u = Du*Lap(u) + A - (B+1)*u + u^2*v,  F_v = Dv*Lap(v) + B*u - u^2*v.
 * Parameter vectors p[4]: FHN (Du, Dv, eps, a); GM (Du, Dv, rho, mu);
 * DIFF (Du, Dv, -, -); BZ (Du, Dv, A, B).
 *
 * Grid: G x G nodes, h = 1/(G-1); field layout [species][y][x], row-major.
 * Discrete Laplacian (App. B.1.1):
 *   Lap(w)_{y,x} = (((w_{y,x+1} + w_{y,x-1}) + w_{y+1,x}) + w_{y-1,x} - 4*w_{y,x}) * (G-1)^2
 * with ghost values equal to the adjacent edge node (mirrored Neumann ghosts).
 * Dividing by h^2 is replaced by multiplying with the exact integer (G-1)^2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "sm64.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the OpenMP loops below use (1 without OpenMP); reported with the
   CPU timings. */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads of the oracle's parallel loops (for
   timing at a given thread count; no effect without OpenMP). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

#define ORC_FHN 0
#define ORC_GM 1
#define ORC_DIFF 2
#define ORC_BZ 3

/* Homogeneous steady state (Sec. 4.1): FHN (0,0); GM (1/mu, 1/mu^2) with
   mu_w = 1, evaluated as u0 = 1/mu, v0 = u0*u0; BZ (A, B/A); DIFF (0,0). */
void orc_equilibrium(int model, const double *p, double *u0, double *v0)
{
    if (model == ORC_GM) {
        double a = 1.0 / p[3];
        *u0 = a;
        *v0 = a * a;
    } else if (model == ORC_BZ) {
        *u0 = p[2];
        *v0 = p[3] / p[2];
    } else {
        *u0 = 0.0;
        *v0 = 0.0;
    }
}

/* Initial state (Sec. 4.1): equilibrium + U(lo, hi) per (realisation,
   species, node).  U = SplitMix64 output number ((r*2 + s)*G*G + node) of
   stream `seed`, top 53 bits times 2^-53.  value = x0 + (lo + (hi-lo)*U)
   in FP64, rounded once to FP32. */
void orc_init_fields(int model, int G, int n_real, const double *p,
                     double lo, double hi, uint64_t seed, float *out)
{
    double x0[2];
    orc_equilibrium(model, p, &x0[0], &x0[1]);
    int64_t cells = (int64_t)G * G;
    for (int64_t r = 0; r < n_real; ++r)
        for (int s = 0; s < 2; ++s)
            for (int64_t c = 0; c < cells; ++c) {
                uint64_t i = ((uint64_t)r * 2u + (uint64_t)s) * (uint64_t)cells + (uint64_t)c;
                double U = orc_u01(seed, i);
                double span = hi - lo;
                double t = span * U;
                double t2 = lo + t;
                double v = x0[s] + t2;
                out[(r * 2 + s) * cells + c] = (float)v;
            }
}

/* Discrete Laplacian of one species field at node (y, x). */
static double lap_at(const double *w, int G, int y, int x)
{
    double c = w[y * G + x];
    double xp = (x + 1 < G) ? w[y * G + x + 1] : c;
    double xm = (x - 1 >= 0) ? w[y * G + x - 1] : c;
    double yp = (y + 1 < G) ? w[(y + 1) * G + x] : c;
    double ym = (y - 1 >= 0) ? w[(y - 1) * G + x] : c;
    double g1 = (double)(G - 1);
    double sum = ((xp + xm) + yp) + ym;
    double c4 = 4.0 * c;
    return (sum - c4) * (g1 * g1);
}

/* Right-hand side F(w) of the method-of-lines system (App. B.1.1) for one
   realisation; w and F are [2][G][G]. */
void orc_rhs(int model, int G, const double *p, const double *w, double *F)
{
    int64_t cells = (int64_t)G * G;
    const double *u = w, *v = w + cells;
    double *Fu = F, *Fv = F + cells;
    for (int y = 0; y < G; ++y)
        for (int x = 0; x < G; ++x) {
            int64_t k = (int64_t)y * G + x;
            double lu = lap_at(u, G, y, x);
            double lv = lap_at(v, G, y, x);
            double du = p[0] * lu;
            double dv = p[1] * lv;
            double ru, rv;
            double uk = u[k], vk = v[k];
            if (model == ORC_FHN) {
                double u3 = (uk * uk) * uk;
                ru = (uk - u3) - vk;
                double av = p[3] * vk;
                rv = p[2] * (uk - av);
            } else if (model == ORC_GM) {
                double uu = uk * uk;
                double q = uu / vk;
                double mu_u = p[3] * uk;
                ru = p[2] * (q - mu_u);
                rv = p[2] * (uu - vk);
            } else if (model == ORC_BZ) {
                double uuv = (uk * uk) * vk;
                double bu = (p[3] + 1.0) * uk;
                ru = (p[2] - bu) + uuv;
                rv = p[3] * uk - uuv;
            } else {
                ru = 0.0;
                rv = 0.0;
            }
            Fu[k] = du + ru;
            Fv[k] = dv + rv;
        }
}

/* Forward Euler (Sec. 5.1): w <- w + dt*F(w), both species from the old
   state, n_steps times, for each of n_real realisations ([n_real][2][G][G]). */
void orc_step(int model, int G, int n_real, const double *p, double dt,
              int64_t n_steps, double *w)
{
    int64_t m = 2 * (int64_t)G * G;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_real; ++r) {
        double *F = (double *)malloc(sizeof(double) * (size_t)m);
        double *wr = w + (int64_t)r * m;
        for (int64_t n = 0; n < n_steps; ++n) {
            orc_rhs(model, G, p, wr, F);
            for (int64_t k = 0; k < m; ++k) {
                double inc = dt * F[k];
                wr[k] = wr[k] + inc;
            }
        }
        free(F);
    }
}

/* Steady-state residual (Sec. 5.1, the L-infinity stopping criterion):
   per realisation, max |F| and sqrt(mean F^2) over both species and all
   nodes, F in FP64 from the given state.  out is [n_real][2]. */
void orc_residual(int model, int G, int n_real, const double *p,
                  const double *w, double *out)
{
    int64_t m = 2 * (int64_t)G * G;
    double *F = (double *)malloc(sizeof(double) * (size_t)m);
    for (int r = 0; r < n_real; ++r) {
        orc_rhs(model, G, p, w + (int64_t)r * m, F);
        double mx = 0.0, ss = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            double a = fabs(F[k]);
            if (a > mx) mx = a;
            ss = ss + F[k] * F[k];
        }
        out[2 * r] = mx;
        out[2 * r + 1] = sqrt(ss / (double)m);
    }
    free(F);
}

/* ---------------------------------------------------------------------
 * Discrete adjoint of forward Euler (gradient of a scalar loss of the final
 * state with respect to the four kinetic/diffusion parameters).  The paper
 * has no gradient; this is the exact reverse-mode derivative of the FP64
 * recursion above, with the initial state held fixed:
 *   lambda_N = dL/dw_N,
 *   g       += dt * (dF/dtheta (w_n))^T lambda_{n+1},
 *   lambda_n = lambda_{n+1} + dt * J_F(w_n)^T lambda_{n+1},   n = N-1..0.
 * The Laplacian with mirrored ghosts is a symmetric matrix, so its transpose
 * is itself.
 * --------------------------------------------------------------------- */

/* y = J_F(w)^T lam and dg[4] = (dF/dtheta(w))^T lam for one realisation. */
/* y = J_F(w)^T lam, dg[i] = lam . dF/dtheta_i(w); dga (nullable) adds the
   magnitudes of the terms of each dg[i] (sum over cells of |term|), a
   measure of how much cancellation the gradient sum holds. */
static void jt_vec_abs(int model, int G, const double *p, const double *w,
                       const double *lam, double *y, double *dg, double *dga)
{
    int64_t cells = (int64_t)G * G;
    const double *u = w, *v = w + cells;
    const double *lu = lam, *lv = lam + cells;
    double *yu = y, *yv = y + cells;
    double g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int yy = 0; yy < G; ++yy)
        for (int x = 0; x < G; ++x) {
            int64_t k = (int64_t)yy * G + x;
            double Llu = lap_at(lu, G, yy, x);
            double Llv = lap_at(lv, G, yy, x);
            double Lu = lap_at(u, G, yy, x);
            double Lv = lap_at(v, G, yy, x);
            double uk = u[k], vk = v[k], a = lu[k], b = lv[k];
            double su, sv;
            g0 = g0 + Lu * a;
            g1 = g1 + Lv * b;
            a0 = a0 + fabs(Lu * a);
            a1 = a1 + fabs(Lv * b);
            if (model == ORC_FHN) {
                double eps = p[2], aa = p[3];
                double duu = 1.0 - 3.0 * (uk * uk);
                su = duu * a + eps * b;
                sv = (-1.0) * a - (eps * aa) * b;
                g2 = g2 + (uk - aa * vk) * b;
                g3 = g3 + (-(eps * vk)) * b;
                a2 = a2 + fabs((uk - aa * vk) * b);
                a3 = a3 + fabs((-(eps * vk)) * b);
            } else if (model == ORC_GM) {
                double rho = p[2], mu = p[3];
                double dfu_du = rho * (2.0 * uk / vk - mu);
                double dfu_dv = -(rho * ((uk * uk) / (vk * vk)));
                double dfv_du = 2.0 * rho * uk;
                double dfv_dv = -rho;
                su = dfu_du * a + dfv_du * b;
                sv = dfu_dv * a + dfv_dv * b;
                g2 = g2 + ((uk * uk) / vk - mu * uk) * a + (uk * uk - vk) * b;
                g3 = g3 + (-(rho * uk)) * a;
                a2 = a2 + fabs(((uk * uk) / vk - mu * uk) * a) + fabs((uk * uk - vk) * b);
                a3 = a3 + fabs((-(rho * uk)) * a);
            } else if (model == ORC_BZ) {
                double B = p[3];
                double dfu_du = -(B + 1.0) + 2.0 * uk * vk;
                double dfu_dv = uk * uk;
                double dfv_du = B - 2.0 * uk * vk;
                double dfv_dv = -(uk * uk);
                su = dfu_du * a + dfv_du * b;
                sv = dfu_dv * a + dfv_dv * b;
                g2 = g2 + a;                          /* dF_u/dA = 1, dF_v/dA = 0 */
                g3 = g3 + (-uk) * a + uk * b;         /* dF_u/dB = -u, dF_v/dB = u */
                a2 = a2 + fabs(a);
                a3 = a3 + fabs((-uk) * a) + fabs(uk * b);
            } else {
                su = 0.0;
                sv = 0.0;
            }
            yu[k] = p[0] * Llu + su;
            yv[k] = p[1] * Llv + sv;
        }
    dg[0] = g0; dg[1] = g1; dg[2] = g2; dg[3] = g3;
    if (dga) {
        dga[0] = a0; dga[1] = a1; dga[2] = a2; dga[3] = a3;
    }
}

static void jt_vec(int model, int G, const double *p, const double *w,
                   const double *lam, double *y, double *dg)
{
    jt_vec_abs(model, G, p, w, lam, y, dg, NULL);
}

/* Reverse sweep for one realisation.  w0: initial state [2][G][G];
   lamN: dL/dw_N (overwritten with dL/dw_0); grad[4] accumulates.
   All n_steps+1 states are stored (plain, memory O(n_steps * 2G^2)). */
int orc_adjoint_one(int model, int G, const double *p, double dt,
                    int64_t n_steps, const double *w0, double *lam,
                    double *grad, double *gabs)
{
    int64_t m = 2 * (int64_t)G * G;
    double *W = (double *)malloc(sizeof(double) * (size_t)m * (size_t)(n_steps + 1));
    double *F = (double *)malloc(sizeof(double) * (size_t)m);
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    if (!W || !F || !y) { free(W); free(F); free(y); return 1; }
    memcpy(W, w0, sizeof(double) * (size_t)m);
    for (int64_t n = 0; n < n_steps; ++n) {
        const double *wn = W + n * m;
        double *wn1 = W + (n + 1) * m;
        orc_rhs(model, G, p, wn, F);
        for (int64_t k = 0; k < m; ++k) wn1[k] = wn[k] + dt * F[k];
    }
    for (int64_t n = n_steps - 1; n >= 0; --n) {
        double dg[4], da[4];
        jt_vec_abs(model, G, p, W + n * m, lam, y, dg, da);
        for (int i = 0; i < 4; ++i) grad[i] = grad[i] + dt * dg[i];
        if (gabs)
            for (int i = 0; i < 4; ++i) gabs[i] = gabs[i] + dt * da[i];
        for (int64_t k = 0; k < m; ++k) lam[k] = lam[k] + dt * y[k];
    }
    free(W); free(F); free(y);
    return 0;
}

/* One step's Jacobian-vector products for the dot-product test:
   jv = J_F(w) dv + (dF/dtheta) dtheta  and  the transpose pair. */
void orc_jvp(int model, int G, const double *p, const double *w,
             const double *dw, const double *dtheta, double *out)
{
    /* Central difference would not be exact; instead linearise by hand. */
    int64_t cells = (int64_t)G * G;
    const double *u = w, *v = w + cells;
    const double *du = dw, *dv = dw + cells;
    for (int yy = 0; yy < G; ++yy)
        for (int x = 0; x < G; ++x) {
            int64_t k = (int64_t)yy * G + x;
            double Ldu = lap_at(du, G, yy, x), Ldv = lap_at(dv, G, yy, x);
            double Lu = lap_at(u, G, yy, x), Lv = lap_at(v, G, yy, x);
            double uk = u[k], vk = v[k], a = du[k], b = dv[k];
            double ou = p[0] * Ldu + dtheta[0] * Lu;
            double ov = p[1] * Ldv + dtheta[1] * Lv;
            if (model == ORC_FHN) {
                double eps = p[2], aa = p[3];
                ou += (1.0 - 3.0 * uk * uk) * a - b;
                ov += eps * (a - aa * b) + dtheta[2] * (uk - aa * vk) + dtheta[3] * (-(eps * vk));
            } else if (model == ORC_GM) {
                double rho = p[2], mu = p[3];
                ou += rho * (2.0 * uk / vk - mu) * a - rho * (uk * uk) / (vk * vk) * b
                      + dtheta[2] * ((uk * uk) / vk - mu * uk) + dtheta[3] * (-(rho * uk));
                ov += 2.0 * rho * uk * a - rho * b + dtheta[2] * (uk * uk - vk);
            } else if (model == ORC_BZ) {
                double B = p[3];
                ou += (-(B + 1.0) + 2.0 * uk * vk) * a + (uk * uk) * b + dtheta[2] - dtheta[3] * uk;
                ov += (B - 2.0 * uk * vk) * a - (uk * uk) * b + dtheta[3] * uk;
            }
            out[k] = ou;
            out[cells + k] = ov;
        }
}

void orc_vjp(int model, int G, const double *p, const double *w,
             const double *lam, double *out_w, double *out_theta)
{
    jt_vec(model, G, p, w, lam, out_w, out_theta);
}

/* Raw generator output, exported so tests can pin it to published values. */
uint64_t orc_sm64(uint64_t seed, uint64_t i) { return orc_sm64_at(seed, i); }
