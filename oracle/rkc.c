/*
 * ORACLE — test infrastructure only.  Plain, slow FP64 reference for the
 * stabilised explicit second-order Runge-Kutta integration of the
 * method-of-lines reaction-diffusion system.  Only tests/, the smoke check
 * and the benchmark's CPU legs may load it.  It shares no code with the
 * CUDA path.  Compiled with -O2 -ffp-contract=off.
 *
 * Paper: arXiv 2203.14742, App. B.2 ("Reaction-diffusion systems"): the RD
 * systems are integrated by ROCK2, an explicit second-order stabilised
 * Runge-Kutta method whose stages follow a three-term recurrence, with the
 * stage number s chosen each step from h_n times a Gershgorin bound of the
 * spectral radius of the Jacobian at w_n, a weighted RMS error norm with
 * absolute and relative tolerances, and a predictive step-size controller
 * with safety factor eta = 0.8.
 *
 * Reading (the paper does not print ROCK2's recurrence coefficients, which
 * are fitted numerically in the method's original publication): the same
 * family's member with closed-form coefficients is used, the second-order
 * Runge-Kutta-Chebyshev method (van der Houwen & Sommeijer 1980; Sommeijer,
 * Shampine & Verwer 1997) with damping eps = 2/13.  With T_j the Chebyshev
 * polynomials of the first kind and
 *   w0 = 1 + eps / s^2,   w1 = T_s'(w0) / T_s''(w0),
 *   b_j = T_j''(w0) / T_j'(w0)^2 (j >= 2),  b_0 = b_1 = b_2,
 *   a_j = 1 - b_j T_j(w0),
 * one step of size h from w_n is
 *   Y_0 = w_n,  Y_1 = Y_0 + mt_1 h F(Y_0),  mt_1 = b_1 w1,
 *   Y_j = (1 - mu_j - nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2}
 *         + mt_j h F(Y_{j-1}) + gt_j h F(Y_0),          j = 2..s,
 *   mu_j = 2 b_j w0 / b_{j-1},  nu_j = -b_j / b_{j-2},
 *   mt_j = 2 b_j w1 / b_{j-1},  gt_j = -a_{j-1} mt_j,
 *   w_{n+1} = Y_s.
 * Applied to w' = lambda w the step multiplies w by
 *   R_s(z) = a_s + b_s T_s(w0 + w1 z),  z = h lambda,
 * which equals 1 + z + z^2/2 + O(z^3) and stays in [-1, 1] for z in
 * [-beta(s), 0], beta(s) = (1 + w0) / w1 (about 0.65 s^2; ROCK2's interval
 * is about 0.81 s^2, hence the paper's rule h rho <= (0.9 s)^2).
 *
 * Readings of the step control (App. B.2, with the points it leaves open):
 *   - rho = the Gershgorin bound max_i sum_j |J_ij| of the Jacobian of F at
 *     w_n, rows taken exactly: a node with n in-domain neighbours (the
 *     mirrored ghost equals the node itself) has diagonal
 *     -n D (G-1)^2 + df/du and off-diagonal sum n D (G-1)^2 + |df/dv|;
 *   - s = the smallest s >= 2 with h rho <= beta(s); if s would exceed
 *     s_max, h is cut to beta(s_max) / rho and s = s_max;
 *   - error estimate of the RKC pair, 2/5 of the trapezoidal-rule defect:
 *       est = (12 (w_n - w_{n+1}) + 6 h (F(w_n) + F(w_{n+1}))) / 15,
 *     which is O(h^3);
 *   - err = sqrt(mean_k (est_k / (atol + rtol max(|w_n,k|, |w_{n+1},k|)))^2)
 *     (the paper's norm, with the square over the whole ratio); the step is
 *     accepted when err <= 1;
 *   - the paper's controller with the exponent matched to the estimate:
 *       fac = eta err^(-1/3) (h_n / h_{n-1}) (err_{n-1} / err)^(1/3)
 *     after an accepted step that follows an accepted step, eta err^(-1/3)
 *     otherwise (first step, or after a rejection; the paper's exponent 1/2
 *     belongs to ROCK2's first-order embedded estimate, and with an O(h^3)
 *     estimate it makes the predictive controller unstable); err is floored
 *     at 1e-10; fac clamped to [0.1, 10], and to at most 1 on the step
 *     after a rejection; h_{n+1} = fac h_n;
 *   - the last step is cut to end exactly at t_end;
 *   - a realisation fails when it needs more than max_attempts attempts or
 *     h drops below 1e-12 t_end.
 * The same driver integrates the 1-D reaction-diffusion-ODE system of
 * rdode.c (model 4), whose realisations are [2][N].
 * RHS evaluations per attempt: s (F(Y_1)..F(Y_{s-1}) and F(Y_s), which is
 * F(w_{n+1}) of the estimate and the next step's F(Y_0)), plus one for the
 * initial F(w_0).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

void orc_rhs(int model, int G, const double *p, const double *w, double *F);
void orc_rdode_rhs(int N, const double *p, const double *w, double *F);
double orc_rdode_gershgorin(int N, const double *p, const double *w);

/* Model 4 is the 1-D reaction-diffusion-ODE system of rdode.c (G = its
   node count N, a realisation is [2][N]); the others are the 2-D systems
   of rd.c ([2][G][G]). */
#define ORC_RDODE 4
static int64_t m_of(int model, int G)
{
    return model == ORC_RDODE ? 2 * (int64_t)G : 2 * (int64_t)G * G;
}
static void rhs_any(int model, int G, const double *p, const double *w, double *F)
{
    if (model == ORC_RDODE) orc_rdode_rhs(G, p, w, F);
    else orc_rhs(model, G, p, w, F);
}

#define RKC_EPS (2.0 / 13.0)

/* Chebyshev T_j, T_j', T_j'' at x for j = 0..s by the three-term
   recurrence T_j = 2x T_{j-1} - T_{j-2} and its first two derivatives. */
static void cheb_at(int s, double x, double *T, double *T1, double *T2)
{
    T[0] = 1.0; T1[0] = 0.0; T2[0] = 0.0;
    T[1] = x;   T1[1] = 1.0; T2[1] = 0.0;
    for (int j = 2; j <= s; ++j) {
        T[j] = 2.0 * x * T[j - 1] - T[j - 2];
        T1[j] = 2.0 * T[j - 1] + 2.0 * x * T1[j - 1] - T1[j - 2];
        T2[j] = 4.0 * T1[j - 1] + 2.0 * x * T2[j - 1] - T2[j - 2];
    }
}

/* Coefficients of the s-stage method (s >= 2): mu, nu, mt, gt indexed by
   stage j (entries 0 and, for mu/nu/gt, 1 unused), plus w0, w1, b_s, a_s
   and beta(s).  ex = {w0, w1, b_s, a_s, beta}. */
void orc_rkc_coef(int s, double *mu, double *nu, double *mt, double *gt, double *ex)
{
    double *T = malloc(sizeof(double) * (size_t)(s + 1));
    double *T1 = malloc(sizeof(double) * (size_t)(s + 1));
    double *T2 = malloc(sizeof(double) * (size_t)(s + 1));
    double *b = malloc(sizeof(double) * (size_t)(s + 1));
    double *a = malloc(sizeof(double) * (size_t)(s + 1));
    const double w0 = 1.0 + RKC_EPS / ((double)s * (double)s);
    cheb_at(s, w0, T, T1, T2);
    const double w1 = T1[s] / T2[s];
    for (int j = 2; j <= s; ++j) b[j] = T2[j] / (T1[j] * T1[j]);
    b[0] = b[2];
    b[1] = b[2];
    for (int j = 0; j <= s; ++j) a[j] = 1.0 - b[j] * T[j];
    for (int j = 0; j <= s; ++j) { mu[j] = 0.0; nu[j] = 0.0; mt[j] = 0.0; gt[j] = 0.0; }
    mt[1] = b[1] * w1;
    for (int j = 2; j <= s; ++j) {
        mu[j] = 2.0 * b[j] * w0 / b[j - 1];
        nu[j] = -b[j] / b[j - 2];
        mt[j] = 2.0 * b[j] * w1 / b[j - 1];
        gt[j] = -a[j - 1] * mt[j];
    }
    ex[0] = w0;
    ex[1] = w1;
    ex[2] = b[s];
    ex[3] = a[s];
    ex[4] = (1.0 + w0) / w1;
    free(T); free(T1); free(T2); free(b); free(a);
}

/* beta(s) = (1 + w0) / w1, the length of the real stability interval. */
double orc_rkc_beta(int s)
{
    double *T = malloc(sizeof(double) * (size_t)(s + 1));
    double *T1 = malloc(sizeof(double) * (size_t)(s + 1));
    double *T2 = malloc(sizeof(double) * (size_t)(s + 1));
    const double w0 = 1.0 + RKC_EPS / ((double)s * (double)s);
    cheb_at(s, w0, T, T1, T2);
    const double beta = (1.0 + w0) / (T1[s] / T2[s]);
    free(T); free(T1); free(T2);
    return beta;
}

/* Partial derivatives (f_u, f_v, g_u, g_v) of the kinetics at (u, v). */
static void kinetics_jac(int model, const double *p, double u, double v, double *J)
{
    if (model == 0) {            /* FHN: f = u - u^3 - v, g = eps (u - a v) */
        J[0] = 1.0 - 3.0 * (u * u);
        J[1] = -1.0;
        J[2] = p[2];
        J[3] = -(p[2] * p[3]);
    } else if (model == 1) {     /* GM: f = rho (u^2/v - mu u), g = rho (u^2 - v) */
        J[0] = p[2] * (2.0 * u / v - p[3]);
        J[1] = -(p[2] * ((u * u) / (v * v)));
        J[2] = p[2] * (2.0 * u);
        J[3] = -p[2];
    } else if (model == 3) {     /* BZ: f = A - (B+1) u + u^2 v, g = B u - u^2 v */
        J[0] = -(p[3] + 1.0) + 2.0 * (u * v);
        J[1] = u * u;
        J[2] = p[3] - 2.0 * (u * v);
        J[3] = -(u * u);
    } else {                     /* DIFF */
        J[0] = 0.0; J[1] = 0.0; J[2] = 0.0; J[3] = 0.0;
    }
}

/* Gershgorin bound of the spectral radius of dF/dw at w ([2][G][G]). */
double orc_gershgorin(int model, int G, const double *p, const double *w)
{
    if (model == ORC_RDODE) return orc_rdode_gershgorin(G, p, w);
    const int64_t cells = (int64_t)G * G;
    const double g2 = (double)(G - 1) * (double)(G - 1);
    const double du = p[0] * g2, dv = p[1] * g2;
    double rho = 0.0;
    for (int y = 0; y < G; ++y)
        for (int x = 0; x < G; ++x) {
            const int64_t k = (int64_t)y * G + x;
            const int n = (x > 0) + (x < G - 1) + (y > 0) + (y < G - 1);
            double J[4];
            kinetics_jac(model, p, w[k], w[cells + k], J);
            const double ru = fabs(-(double)n * du + J[0]) + (double)n * du + fabs(J[1]);
            const double rv = fabs(-(double)n * dv + J[3]) + (double)n * dv + fabs(J[2]);
            if (ru > rho) rho = ru;
            if (rv > rho) rho = rv;
        }
    return rho;
}

/* One step of size h with s stages (s >= 2) of one realisation w [2][G][G];
   F0 = F(w) on entry.  On return w = w_{n+1} and, if Fs is non-null,
   Fs = F(w_{n+1}).  Work buffers: 3 arrays of m doubles. */
static void rkc_step_one(int model, int G, const double *p, double h, int s,
                         const double *mu, const double *nu, const double *mt, const double *gt,
                         double *w, const double *F0, double *Fs, double *Ym2, double *Ym1, double *Fj)
{
    const int64_t m = m_of(model, G);
    for (int64_t k = 0; k < m; ++k) {
        Ym2[k] = w[k];
        Ym1[k] = w[k] + (mt[1] * h) * F0[k];
    }
    for (int j = 2; j <= s; ++j) {
        rhs_any(model, G, p, Ym1, Fj);
        const double c0 = (1.0 - mu[j]) - nu[j];
        const double cf = mt[j] * h, c0f = gt[j] * h;
        for (int64_t k = 0; k < m; ++k) {
            double y = c0 * w[k];
            y = y + mu[j] * Ym1[k];
            y = y + nu[j] * Ym2[k];
            y = y + cf * Fj[k];
            y = y + c0f * F0[k];
            Ym2[k] = Ym1[k];
            Ym1[k] = y;
        }
    }
    memcpy(w, Ym1, sizeof(double) * (size_t)m);
    if (Fs) rhs_any(model, G, p, w, Fs);
}

/* Fixed schedule: n_steps steps of size h with s stages each, for n_real
   realisations w [n_real][2][G][G] (no error control). */
void orc_rkc_fixed(int model, int G, int n_real, const double *p, double h, int s,
                   int64_t n_steps, double *w)
{
    const int64_t m = m_of(model, G);
    double *mu = malloc(sizeof(double) * (size_t)(s + 1)), *nu = malloc(sizeof(double) * (size_t)(s + 1));
    double *mt = malloc(sizeof(double) * (size_t)(s + 1)), *gt = malloc(sizeof(double) * (size_t)(s + 1));
    double ex[5];
    orc_rkc_coef(s, mu, nu, mt, gt, ex);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_real; ++r) {
        double *buf = malloc(sizeof(double) * (size_t)(5 * m));
        double *F0 = buf, *Fs = buf + m, *a = buf + 2 * m, *b = buf + 3 * m, *c = buf + 4 * m;
        double *wr = w + (int64_t)r * m;
        rhs_any(model, G, p, wr, F0);
        for (int64_t n = 0; n < n_steps; ++n) {
            rkc_step_one(model, G, p, h, s, mu, nu, mt, gt, wr, F0, Fs, a, b, c);
            memcpy(F0, Fs, sizeof(double) * (size_t)m);
        }
        free(buf);
    }
    free(mu); free(nu); free(mt); free(gt);
}

/* Adaptive integration from t = 0 to t_end (App. B.2 with the readings
   above) of n_real realisations w [n_real][2][G][G].  h0: first trial step.
   stats [n_real][4]: accepted steps, rejected steps, RHS evaluations,
   largest s.  Returns the number of realisations that failed (their state
   is left where the control gave up). */
int orc_rkc_adaptive(int model, int G, int n_real, const double *p, double t_end, double h0,
                     double rtol, double atol, int s_max, int64_t max_attempts, double *w,
                     int64_t *stats)
{
    const int64_t m = m_of(model, G);
    const double eta = 0.8;
    int failed = 0;
    /* coefficient tables for every s = 2..s_max, and beta(s) */
    const int64_t stride = s_max + 1;
    double *tab = malloc(sizeof(double) * (size_t)(4 * stride * stride));
    double *beta = malloc(sizeof(double) * (size_t)stride);
    for (int s = 2; s <= s_max; ++s) {
        double ex[5];
        double *row = tab + 4 * stride * s;
        orc_rkc_coef(s, row, row + stride, row + 2 * stride, row + 3 * stride, ex);
        beta[s] = ex[4];
    }
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : failed)
    for (int r = 0; r < n_real; ++r) {
        double *buf = malloc(sizeof(double) * (size_t)(6 * m));
        double *F0 = buf, *Fs = buf + m, *a = buf + 2 * m, *b = buf + 3 * m, *c = buf + 4 * m;
        double *wn = buf + 5 * m;
        double *wr = w + (int64_t)r * m;
        int64_t *st = stats + 4 * (int64_t)r;
        st[0] = 0; st[1] = 0; st[2] = 1; st[3] = 0;
        rhs_any(model, G, p, wr, F0);
        double t = 0.0, h = h0, h_prev = 0.0, err_prev = 0.0;
        int have_prev = 0, after_reject = 0, ok = 1;
        int64_t attempts = 0;
        while (t < t_end) {
            if (attempts >= max_attempts || h < 1e-12 * t_end) { ok = 0; break; }
            attempts = attempts + 1;
            int last = 0;
            if (h >= t_end - t) { h = t_end - t; last = 1; }
            const double rho = orc_gershgorin(model, G, p, wr);
            int s = 2;
            while (s < s_max && h * rho > beta[s]) s = s + 1;
            if (h * rho > beta[s]) { h = beta[s_max] / rho; last = 0; }
            const double *row = tab + 4 * stride * s;
            memcpy(wn, wr, sizeof(double) * (size_t)m);
            rkc_step_one(model, G, p, h, s, row, row + stride, row + 2 * stride, row + 3 * stride,
                         wn, F0, Fs, a, b, c);
            st[2] = st[2] + s;
            if (s > st[3]) st[3] = s;
            double sum = 0.0;
            for (int64_t k = 0; k < m; ++k) {
                const double e = (12.0 * (wr[k] - wn[k]) + 6.0 * h * (F0[k] + Fs[k])) / 15.0;
                const double aw = fabs(wr[k]), an = fabs(wn[k]);
                const double sc = atol + rtol * (aw > an ? aw : an);
                const double q = e / sc;
                sum = sum + q * q;
            }
            const double err = sqrt(sum / (double)m);
            if (!isfinite(err)) { ok = 0; break; }
            const double ef = err > 1e-10 ? err : 1e-10;
            double fac;
            if (err <= 1.0) {
                t = last ? t_end : t + h;
                memcpy(wr, wn, sizeof(double) * (size_t)m);
                memcpy(F0, Fs, sizeof(double) * (size_t)m);
                st[0] = st[0] + 1;
                fac = eta * pow(ef, -1.0 / 3.0);
                if (have_prev)
                    fac = fac * (h / h_prev) * pow(err_prev / ef, 1.0 / 3.0);
                if (fac < 0.1) fac = 0.1;
                if (fac > 10.0) fac = 10.0;
                if (after_reject && fac > 1.0) fac = 1.0;
                h_prev = h;
                err_prev = ef;
                have_prev = 1;
                after_reject = 0;
            } else {
                st[1] = st[1] + 1;
                fac = eta * pow(ef, -1.0 / 3.0);
                if (fac < 0.1) fac = 0.1;
                if (fac > 10.0) fac = 10.0;
                after_reject = 1;
            }
            h = fac * h;
        }
        if (!ok) failed = failed + 1;
        free(buf);
    }
    free(tab);
    free(beta);
    return failed;
}
