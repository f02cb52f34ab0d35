/*
 * ORACLE — test infrastructure only.  Plain, slow FP64 reference for the
 * correlation-integral part of the CIL hot path.  Only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code
 * with the CUDA path.  Compiled with -O2 -ffp-contract=off.
 *
 * Paper: arXiv 2203.14742.
 *   Correlation sum C(R, s, s~) with strict '<', eq. (eCDF), Sec. 2.1;
 *   CIL vector y_m = C(R_m, s^k, s^l), eq. (CIL); power-law radii
 *   R_m = R0 * b^-m with R0 the largest distance, Sec. 2.1 and Sec. 3.2;
 *   mean / covariance of y over set pairs, Alg. 1 step 3;
 *   bootstrap resampling with replacement of each half, Alg. 5 (appendix A)
 *   and Alg. 6; cost f = (y - mu)^T Sigma^-1 (y - mu), eq. (cil:CF) and
 *   eq. (cil:CF_synth).
 *
 * Readings of points the paper leaves open (each stated where used):
 *   - distance = plain Euclidean norm of the difference vector; its square
 *     is the exact real sum of squared differences of the FP32 inputs,
 *     rounded once to the nearest double (see d2_f32), so no evaluation
 *     order enters;
 *   - R_k = R_{k-1} / b in FP64 (k = 1..M), thresholds T_k = R_k * R_k, and
 *     "d < R_k" is decided as d^2 < T_k;
 *   - the linear law of Sec. 2.1 (R_k = R0 - k h, h = (R0 - R_M) / M,
 *     R_M = the smallest cross-set distance, Table 1 for the MC and RD-ODE
 *     models) as the FP64 expressions h = (R0 - R_M) / M, R_k = R0 - k h;
 *   - covariance normaliser 1/(T-1);
 *   - components whose count is identical across all resamples are
 *     inactive; the Gaussian statistics use the active block only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "sm64.h"

int orc_adjoint_one(int model, int G, const double *p, double dt,
                    int64_t n_steps, const double *w0, double *lam,
                    double *grad, double *gabs);
void orc_step(int model, int G, int n_real, const double *p, double dt,
              int64_t n_steps, double *w);

/* Squared distance of two FP32 patterns (eq. eCDF, Sec. 2.1).  The paper
   defines the distance on the reals; the value used here is that real
   number, S = sum_t (x_t - y_t)^2 of the given FP32 values, formed exactly
   and rounded once to the nearest double (ties to even).  It depends on no
   evaluation order.

   How it is formed exactly.  A finite float is m 2^e with an integer
   |m| < 2^24 and e >= -149 (e = -149 for subnormals).  Each term
   (x - y)^2 = x^2 + y^2 - 2 x y is then three integers below 2^48 times
   powers of two 2^p with p >= -298.  The integers are added, exactly, into
   one counter c_p per power of two (128-bit, so no counter can overflow),
   giving S = sum_p c_p 2^p.  The binary digits of N = S 2^298 follow by
   carrying from the lowest power upward (digit = c mod 2, carry = the
   rest halved), and N is rounded to 53 significant bits.  A non-finite
   input element gives NaN. */
#define XP_OFFSET 298           /* counter index = p + 298 >= 0 */
#define XP_COUNTERS 512         /* p + 298 <= 2 * 104 + 1 + 298 = 507 */
#define XP_BITS 640             /* N < 2^(555 + 33) for d < 2^31 */

/* float -> (signed integer significand, exponent); returns 0 if not finite */
static int float_parts(float f, int64_t *m, int *e)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    const int ef = (int)((u >> 23) & 0xffu);
    int64_t mm = (int64_t)(u & 0x7fffffu);
    if (ef == 0xff) return 0;
    if (ef != 0) {
        mm += (int64_t)1 << 23;
        *e = ef - 150;
    } else {
        *e = -149;
    }
    *m = (u >> 31) ? -mm : mm;
    return 1;
}

static double d2_f32(const float *x, const float *y, int64_t d)
{
    __int128 c[XP_COUNTERS];
    for (int k = 0; k < XP_COUNTERS; ++k) c[k] = 0;
    for (int64_t t = 0; t < d; ++t) {
        int64_t mx, my;
        int ex, ey;
        if (!float_parts(x[t], &mx, &ex) || !float_parts(y[t], &my, &ey)) return NAN;
        c[2 * ex + XP_OFFSET] += mx * mx;              /* x^2 */
        c[2 * ey + XP_OFFSET] += my * my;              /* y^2 */
        c[ex + ey + 1 + XP_OFFSET] -= mx * my;         /* -2 x y */
    }
    /* binary digits of N = sum_k c[k] 2^k */
    unsigned char bit[XP_BITS];
    __int128 carry = 0;
    for (int k = 0; k < XP_BITS; ++k) {
        const __int128 t = carry + (k < XP_COUNTERS ? c[k] : 0);
        const int digit = (t % 2) != 0;        /* t mod 2 in {0, 1} (t % 2 may be -1) */
        bit[k] = (unsigned char)digit;
        carry = (t - digit) / 2;               /* exact: t = 2 carry + digit */
    }
    if (carry != 0) return NAN;   /* cannot happen: S >= 0 and N < 2^640 */
    /* round N to 53 significant bits, ties to even */
    int p = -1;
    for (int i = XP_BITS - 1; i >= 0 && p < 0; --i)
        if (bit[i]) p = i;
    if (p < 0) return 0.0;
    const int low = p > 52 ? p - 52 : 0;   /* lowest kept bit */
    uint64_t mant = 0;
    for (int i = p; i >= low; --i) mant = 2 * mant + bit[i];
    if (low > 0) {
        const int half = bit[low - 1];
        int sticky = 0;
        for (int i = low - 2; i >= 0; --i) sticky |= bit[i];
        if (half && (sticky || (mant & 1u))) mant += 1;   /* may reach 2^53: still exact */
    }
    return ldexp((double)mant, low - XP_OFFSET);
}

/* The squared distance, for the other oracle files. */
double orc_d2_exact(const float *x, const float *y, int64_t d)
{
    return d2_f32(x, y, d);
}

static double d2_f64(const double *x, const double *y, int64_t d)
{
    double acc = 0.0;
    for (int64_t t = 0; t < d; ++t) {
        double df = x[t] - y[t];
        double sq = df * df;
        acc = acc + sq;
    }
    return acc;
}

/* All cross-set squared distances: d2[i*n2 + j] = ||X1_i - X2_j||^2. */
void orc_pair_d2(const float *X1, int64_t n1, const float *X2, int64_t n2,
                 int64_t d, double *d2)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n1; ++i)
        for (int64_t j = 0; j < n2; ++j)
            d2[i * n2 + j] = d2_f32(X1 + i * d, X2 + j * d, d);
}

/* Radii (Sec. 2.1): R0 = sqrt(max d^2) over the given pairs,
   R_k = R_{k-1} / b for k = 1..M.  radii[0..M-1] = R_1..R_M.  Returns R0. */
double orc_radii(const double *d2, int64_t n_pairs, double b, int M, double *radii)
{
    double mx = 0.0;
    for (int64_t k = 0; k < n_pairs; ++k)
        if (d2[k] > mx) mx = d2[k];
    double R = sqrt(mx);
    double R0 = R;
    for (int k = 0; k < M; ++k) {
        R = R / b;
        radii[k] = R;
    }
    return R0;
}

/* Linear radii law (Sec. 2.1, Sec. 3.2; Table 1 uses it for the MC and
   RD-ODE models): R0 = sqrt(max d^2) and R_M = sqrt(min d^2) over the given
   pairs (the largest and the smallest distance), h = (R0 - R_M) / M,
   R_k = R0 - k h for k = 1..M (each an FP64 expression, k exact).
   radii[0..M-1] = R_1..R_M.  Returns R0; *Rmin receives sqrt(min d^2). */
double orc_radii_linear(const double *d2, int64_t n_pairs, int M, double *radii, double *Rmin)
{
    double mx = d2[0], mn = d2[0];
    for (int64_t k = 1; k < n_pairs; ++k) {
        if (d2[k] > mx) mx = d2[k];
        if (d2[k] < mn) mn = d2[k];
    }
    const double R0 = sqrt(mx);
    const double RM = sqrt(mn);
    const double h = (R0 - RM) / (double)M;
    for (int k = 1; k <= M; ++k) {
        const double kh = (double)k * h;
        radii[k - 1] = R0 - kh;
    }
    *Rmin = RM;
    return R0;
}

/* Power law with the decay fitted to the range of the distances (Sec. 2.1,
   Sec. 3.2; Table 1 uses it for the FHN, GM and BZ models): R0 = sqrt(max
   d^2), R_min = sqrt(min d^2), b > 1 with R_M / R0 = b^-M, R_k = R_{k-1} / b.
   Reading (the paper gives the condition, not how b is computed): b is the
   smallest double whose M-th power, formed as M - 1 sequential products
   each rounded to nearest, reaches c = R0 / R_min, found by halving
   [1, c] (mid = lo + (hi - lo) * 0.5, every operation rounded to nearest)
   until lo and hi are adjacent; b = 1 when c <= 1 (R_min = R0) and b = +inf
   when c is not finite (R_min = 0), where every R_k = R0 / b^k is 0. */
double orc_fitted_b(double c, int M)
{
    if (!(c < INFINITY)) return INFINITY;
    if (!(c > 1.0)) return 1.0;
    double lo = 1.0, hi = c;
    for (int it = 0; it < 400; ++it) {
        const double half = (hi - lo) * 0.5;
        const double mid = lo + half;
        if (!(mid > lo) || !(mid < hi)) break;
        double p = mid;
        for (int k = 1; k < M; ++k) p = p * mid;
        if (p < c) lo = mid;
        else hi = mid;
    }
    return hi;
}

/* radii[0..M-1] = R_1..R_M of the fitted power law; returns R0, *b_out = b */
double orc_radii_fitted(const double *d2, int64_t n_pairs, int M, double *radii, double *b_out)
{
    double mx = d2[0], mn = d2[0];
    for (int64_t k = 1; k < n_pairs; ++k) {
        if (d2[k] > mx) mx = d2[k];
        if (d2[k] < mn) mn = d2[k];
    }
    const double R0 = sqrt(mx), Rm = sqrt(mn);
    const double b = orc_fitted_b(R0 / Rm, M);
    double R = R0;
    for (int k = 0; k < M; ++k) {
        R = R / b;
        radii[k] = R;
    }
    *b_out = b;
    return R0;
}

/* Bin index K_ij = #{k in 1..M : d_ij < R_k} (strict, eq. eCDF), and
   counts[k-1] = #{(i,j) : K_ij >= k} = N1*N2 * C(R_k). */
void orc_bins_counts(const double *d2, int64_t n_pairs, const double *radii,
                     int M, uint8_t *bins, int64_t *counts)
{
    for (int k = 0; k < M; ++k) counts[k] = 0;
    for (int64_t q = 0; q < n_pairs; ++q) {
        int K = 0;
        for (int k = 0; k < M; ++k) {
            double T = radii[k] * radii[k];
            if (d2[q] < T) K = K + 1;
        }
        bins[q] = (uint8_t)K;
        for (int k = 0; k < K; ++k) counts[k] += 1;
    }
}

/* Bootstrap indices (Alg. 5 step 2.1): resample t draws n1 indices into
   set 1 and n2 into set 2, with replacement.  Index a of side s in resample
   t is SplitMix64 output number ((t*2 + s) << 32 | a) of stream `seed`,
   mapped to [0, n) by Lemire's multiply-shift. */
void orc_bootstrap_indices(uint64_t seed, int T, int64_t n1, int64_t n2,
                           int32_t *I, int32_t *J)
{
    for (int t = 0; t < T; ++t) {
        for (int64_t a = 0; a < n1; ++a) {
            uint64_t ctr = (((uint64_t)t * 2u + 0u) << 32) | (uint64_t)a;
            I[(int64_t)t * n1 + a] = (int32_t)orc_index(seed, ctr, (uint32_t)n1);
        }
        for (int64_t b = 0; b < n2; ++b) {
            uint64_t ctr = (((uint64_t)t * 2u + 1u) << 32) | (uint64_t)b;
            J[(int64_t)t * n2 + b] = (int32_t)orc_index(seed, ctr, (uint32_t)n2);
        }
    }
}

/* Correlation counts of resampled set pairs: for each resample t,
   Y[t][k-1] = sum_a sum_b [K_{I_a, J_b} >= k]  (the numerator of eq. eCDF
   for the resampled sets s^1 = X1[I], s^2 = X2[J]). */
void orc_resample_counts(const uint8_t *bins, int64_t n1, int64_t n2, int M,
                         int T, const int32_t *I, const int32_t *J, int64_t *Y)
{
    for (int t = 0; t < T; ++t) {
        int64_t *y = Y + (int64_t)t * M;
        for (int k = 0; k < M; ++k) y[k] = 0;
        for (int64_t a = 0; a < n1; ++a)
            for (int64_t b = 0; b < n2; ++b) {
                int K = bins[(int64_t)I[(int64_t)t * n1 + a] * n2 + J[(int64_t)t * n2 + b]];
                /* y[k-1] counts [K >= k] for k = 1..M only */
                for (int k = 0; k < K && k < M; ++k) y[k] += 1;
            }
    }
}

/* Synthetic-likelihood statistics (Alg. 1 step 3, eq. cil:CF, eq.
   cil:CF_synth).  y_t = Y_t / n_pairs, n_pairs = n1*n2.  The mean and the
   sample covariance (normaliser 1/(T-1)) of the y_t are rational numbers of
   the integer counts; they are formed exactly from S_k = sum_t Y[t][k] and
   P_kl = sum_t Y[t][k] Y[t][l] and rounded at the end:
     mu_k     = S_k / (T n_pairs),
     Sigma_kl = (T P_kl - S_k S_l) / (T (T-1) n_pairs^2)
   (numerator and denominator exact 64-bit integers, each converted to FP64
   with rounding to nearest, then one FP64 division).
   active[k] = 1 unless all Y[t][k] are equal;
   L = lower Cholesky factor of the active block (Cholesky-Banachiewicz);
   logdet = 2*sum log L_ii; f = || L^-1 (y_obs - mu)_act ||^2;
   loglik = -(f + logdet + M_act*log(2*pi))/2.
   cov and chol are M x M; chol holds the factor of the active block packed
   into its leading M_act x M_act corner.  Returns 0, or 3 when the active
   block is not positive definite.  Requires T^2 n_pairs^2 < 2^62. */
int orc_stats(const int64_t *Y, int T, int M, int64_t n_pairs,
              const double *y_obs, double *mu, double *cov, double *chol,
              double *logdet, double *f, double *loglik, uint8_t *active,
              int *m_act_out)
{
    int64_t S[256];
    for (int k = 0; k < M; ++k) {
        int64_t s = 0;
        for (int t = 0; t < T; ++t) s += Y[(int64_t)t * M + k];
        S[k] = s;
        mu[k] = (double)s / ((double)T * (double)n_pairs);
        int same = 1;
        for (int t = 1; t < T; ++t)
            if (Y[(int64_t)t * M + k] != Y[k]) same = 0;
        active[k] = (uint8_t)(same ? 0 : 1);
    }
    const int64_t den = (int64_t)T * (int64_t)(T - 1) * n_pairs * n_pairs;
    for (int k = 0; k < M; ++k)
        for (int l = 0; l < M; ++l) {
            int64_t P = 0;
            for (int t = 0; t < T; ++t) P += Y[(int64_t)t * M + k] * Y[(int64_t)t * M + l];
            const int64_t num = (int64_t)T * P - S[k] * S[l];
            cov[k * M + l] = (double)num / (double)den;
        }
    int idx[256];
    int ma = 0;
    for (int k = 0; k < M; ++k)
        if (active[k]) idx[ma++] = k;
    *m_act_out = ma;
    for (int q = 0; q < M * M; ++q) chol[q] = 0.0;
    int status = 0;
    for (int i = 0; i < ma && status == 0; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = cov[idx[i] * M + idx[j]];
            for (int k = 0; k < j; ++k) s = s - chol[i * M + k] * chol[j * M + k];
            if (i == j) {
                if (!(s > 0.0)) { status = 3; break; }
                chol[i * M + i] = sqrt(s);
            } else {
                chol[i * M + j] = s / chol[j * M + j];
            }
        }
    }
    double ld = 0.0;
    if (status == 0)
        for (int i = 0; i < ma; ++i) ld = ld + log(chol[i * M + i]);
    *logdet = status == 0 ? 2.0 * ld : NAN;
    if (y_obs && status == 0) {
        double z[256];
        double ff = 0.0;
        for (int i = 0; i < ma; ++i) {
            double s = y_obs[idx[i]] - mu[idx[i]];
            for (int k = 0; k < i; ++k) s = s - chol[i * M + k] * z[k];
            z[i] = s / chol[i * M + i];
            ff = ff + z[i] * z[i];
        }
        *f = ff;
        *loglik = -0.5 * (ff + *logdet + (double)ma * log(2.0 * 3.14159265358979323846));
    } else {
        *f = NAN;
        *loglik = NAN;
    }
    return status;
}

/* ---------------------------------------------------------------------
 * Smoothed correlation integral (the paper has no gradient; this is the
 * differentiable surrogate whose gradient informs proposals):
 *   C_k = (1/(n1 n2)) sum_ij sigma((R_k - d_ij)/tau_k),  tau_k = tau_frac*R_k,
 *   sigma(z) = 1/(1+exp(-z)),  d_ij = sqrt(d^2_ij) (sequential FP64 sum).
 * loss = sum_k cot_k C_k.  gX1/gX2 = d loss / d patterns (may be NULL).
 * --------------------------------------------------------------------- */
void orc_smooth_cil(const double *X1, int64_t n1, const double *X2, int64_t n2,
                    int64_t d, const double *radii, int M, double tau_frac,
                    const double *cot, double *C, double *gX1, double *gX2)
{
    for (int k = 0; k < M; ++k) C[k] = 0.0;
    if (gX1) memset(gX1, 0, sizeof(double) * (size_t)(n1 * d));
    if (gX2) memset(gX2, 0, sizeof(double) * (size_t)(n2 * d));
    double inv = 1.0 / ((double)n1 * (double)n2);
    for (int64_t i = 0; i < n1; ++i)
        for (int64_t j = 0; j < n2; ++j) {
            const double *x = X1 + i * d, *y = X2 + j * d;
            double dd = sqrt(d2_f64(x, y, d));
            double wsum = 0.0; /* d loss / d d_ij */
            for (int k = 0; k < M; ++k) {
                double tau = tau_frac * radii[k];
                double z = (radii[k] - dd) / tau;
                double s = 1.0 / (1.0 + exp(-z));
                C[k] = C[k] + s * inv;
                /* d sigma / d d = -sigma(1-sigma)/tau */
                wsum = wsum + cot[k] * (-(s * (1.0 - s)) / tau) * inv;
            }
            if ((gX1 || gX2) && dd > 0.0) {
                double c = wsum / dd; /* d d / d x = (x - y)/d */
                for (int64_t t = 0; t < d; ++t) {
                    double g = c * (x[t] - y[t]);
                    if (gX1) gX1[i * d + t] += g;
                    if (gX2) gX2[j * d + t] -= g;
                }
            }
        }
}

/* Gradient of loss = sum_k cot_k C_k(patterns(w_N(theta))) with respect to
   theta[4], by the FP64 discrete adjoint.  w0: initial states of n_real
   realisations [n_real][2][G][G] (held fixed); set1/set2: realisation
   indices of the two pattern sets; species_mask: bit0 = u, bit1 = v (the
   pattern is the concatenation of the selected species fields).
   Radii are held fixed.  C_out[M] receives the forward value. */
int orc_smooth_cil_grad(int model, int G, int n_real, const double *p,
                        double dt, int64_t n_steps, const double *w0,
                        int species_mask, const int32_t *set1, int64_t n1,
                        const int32_t *set2, int64_t n2, const double *radii,
                        int M, double tau_frac, const double *cot,
                        double *C_out, double *grad, double *gabs)
{
    int64_t cells = (int64_t)G * G, m = 2 * cells;
    int nsp = ((species_mask & 1) ? 1 : 0) + ((species_mask & 2) ? 1 : 0);
    int64_t d = nsp * cells;
    double *W = (double *)malloc(sizeof(double) * (size_t)(m * n_real));
    memcpy(W, w0, sizeof(double) * (size_t)(m * n_real));
    orc_step(model, G, n_real, p, dt, n_steps, W);
    double *X1 = (double *)malloc(sizeof(double) * (size_t)(n1 * d));
    double *X2 = (double *)malloc(sizeof(double) * (size_t)(n2 * d));
    double *g1 = (double *)malloc(sizeof(double) * (size_t)(n1 * d));
    double *g2 = (double *)malloc(sizeof(double) * (size_t)(n2 * d));
    for (int pass = 0; pass < 2; ++pass) {
        const int32_t *set = pass ? set2 : set1;
        int64_t n = pass ? n2 : n1;
        double *X = pass ? X2 : X1;
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = 0;
            for (int s = 0; s < 2; ++s)
                if (species_mask & (1 << s)) {
                    memcpy(X + i * d + o, W + (int64_t)set[i] * m + s * cells, sizeof(double) * (size_t)cells);
                    o += cells;
                }
        }
    }
    orc_smooth_cil(X1, n1, X2, n2, d, radii, M, tau_frac, cot, C_out, g1, g2);
    /* lambda_N per realisation: scatter pattern gradients into the state. */
    double *lam = (double *)calloc((size_t)(m * n_real), sizeof(double));
    for (int pass = 0; pass < 2; ++pass) {
        const int32_t *set = pass ? set2 : set1;
        int64_t n = pass ? n2 : n1;
        double *g = pass ? g2 : g1;
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = 0;
            for (int s = 0; s < 2; ++s)
                if (species_mask & (1 << s)) {
                    double *dst = lam + (int64_t)set[i] * m + s * cells;
                    for (int64_t c = 0; c < cells; ++c) dst[c] += g[i * d + o + c];
                    o += cells;
                }
        }
    }
    for (int i = 0; i < 4; ++i) grad[i] = 0.0;
    if (gabs)
        for (int i = 0; i < 4; ++i) gabs[i] = 0.0;
    int rc = 0;
    double *gr = (double *)calloc((size_t)(4 * n_real), sizeof(double));
    double *ga = (double *)calloc((size_t)(4 * n_real), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_real; ++r) {
        int nz = 0;
        for (int64_t k = 0; k < m; ++k)
            if (lam[(int64_t)r * m + k] != 0.0) { nz = 1; break; }
        if (!nz) continue;
        if (orc_adjoint_one(model, G, p, dt, n_steps, w0 + (int64_t)r * m,
                            lam + (int64_t)r * m, gr + 4 * r, ga + 4 * r))
            rc = 1;
    }
    for (int r = 0; r < n_real; ++r)
        for (int i = 0; i < 4; ++i) {
            grad[i] = grad[i] + gr[4 * r + i];
            if (gabs) gabs[i] = gabs[i] + ga[4 * r + i];
        }
    free(gr); free(ga); free(lam); free(W); free(X1); free(X2); free(g1); free(g2);
    return rc;
}

/* Loss value only (for finite differences). */
double orc_smooth_cil_loss(int model, int G, int n_real, const double *p,
                           double dt, int64_t n_steps, const double *w0,
                           int species_mask, const int32_t *set1, int64_t n1,
                           const int32_t *set2, int64_t n2, const double *radii,
                           int M, double tau_frac, const double *cot, double *C_out)
{
    int64_t cells = (int64_t)G * G, m = 2 * cells;
    int nsp = ((species_mask & 1) ? 1 : 0) + ((species_mask & 2) ? 1 : 0);
    int64_t d = nsp * cells;
    double *W = (double *)malloc(sizeof(double) * (size_t)(m * n_real));
    memcpy(W, w0, sizeof(double) * (size_t)(m * n_real));
    orc_step(model, G, n_real, p, dt, n_steps, W);
    double *X1 = (double *)malloc(sizeof(double) * (size_t)(n1 * d));
    double *X2 = (double *)malloc(sizeof(double) * (size_t)(n2 * d));
    for (int pass = 0; pass < 2; ++pass) {
        const int32_t *set = pass ? set2 : set1;
        int64_t n = pass ? n2 : n1;
        double *X = pass ? X2 : X1;
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = 0;
            for (int s = 0; s < 2; ++s)
                if (species_mask & (1 << s)) {
                    memcpy(X + i * d + o, W + (int64_t)set[i] * m + s * cells, sizeof(double) * (size_t)cells);
                    o += cells;
                }
        }
    }
    orc_smooth_cil(X1, n1, X2, n2, d, radii, M, tau_frac, cot, C_out, NULL, NULL);
    double L = 0.0;
    for (int k = 0; k < M; ++k) L = L + cot[k] * C_out[k];
    free(W); free(X1); free(X2);
    return L;
}
