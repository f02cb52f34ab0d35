// Step control of the stabilised second-order Runge-Kutta integrator
// (App. B.2), shared by the 2-D kernel (rkc.cu, thread 0 of a CTA owns the
// state in shared memory) and the 1-D kernel (rkc1d.cu, every lane of a
// warp holds an identical copy in registers).  Coefficient tables:
// rkc_tables_fill() forms tab[s][j] = (mu_j, nu_j, mt_j, gt_j) (FP32,
// s = 2..RD_RKC_S_MAX, j = 1..s) and beta[s] (FP64) into memory the handle
// owns (rd_init, once per handle and so per device).
#pragma once
#include "common.cuh"
#include "tile.cuh"

namespace rdcil {

constexpr int RKC_SMAX = RD_RKC_S_MAX;
constexpr int RKC_STRIDE = RKC_SMAX + 1;


// Step control state of one realisation.
struct RkcCtl {
    double t, t_end, h, h_prev;
    int64_t attempts, n_acc, n_rej, n_rhs;
    float err_prev, hf, rho, rho_new;
    int s, s_used, last, have_prev, after_reject, accept, done, fail;
};

struct RkcRun {
    double t_end, h0, rtol, atol;
    int32_t s_max, s_fixed;
    int64_t n_fixed, max_attempts;
};

// Plan the next attempt (thread 0): clip to t_end, pick s from rho.
__device__ __forceinline__ void rkc_plan(RkcCtl &c, const RkcRun &run, const double *__restrict__ beta) {
    if (run.s_fixed >= 2) {
        if (c.n_acc >= run.n_fixed) { c.done = 1; return; }
        c.h = run.h0;
        c.s = run.s_fixed;
    } else {
        if (!(c.t < c.t_end)) { c.done = 1; return; }
        if (c.attempts >= run.max_attempts || c.h < 1e-12 * c.t_end) { c.done = 1; c.fail = 1; return; }
        c.last = 0;
        if (c.h >= c.t_end - c.t) { c.h = c.t_end - c.t; c.last = 1; }
        const double hr = c.h * (double)c.rho;
        // beta(s) < 0.66 s^2 for every s, so no s below sqrt(hr / 0.66)
        // qualifies: start the search for the smallest s there
        int s = (int)sqrtf((float)hr / 0.66f);
        s = s < 2 ? 2 : (s > run.s_max ? run.s_max : s);
        while (s < run.s_max && hr > beta[s]) ++s;
        if (hr > beta[s]) { c.h = beta[run.s_max] / (double)c.rho; c.last = 0; }
        c.s = s;
    }
    c.attempts += 1;
    c.hf = (float)c.h;
    c.n_rhs += c.s;
    if (c.s > c.s_used) c.s_used = c.s;
}

// Accept or reject the attempt just made (thread 0), then plan the next.
// The step-size factor is computed in FP32 (the FP32 error estimate it
// comes from is far less precise than that); t and h stay FP64.
__device__ __forceinline__ void rkc_decide(RkcCtl &c, const RkcRun &run, const double *__restrict__ beta,
                                           float sumsq, int m) {
    if (run.s_fixed >= 2) {
        c.accept = 1;
        c.n_acc += 1;
        rkc_plan(c, run, beta);
        return;
    }
    const float err = sqrtf(sumsq / (float)m);
    if (!isfinite(err)) { c.accept = 0; c.done = 1; c.fail = 2; return; }
    const float ef = fmaxf(err, 1e-10f);
    float fac;
    if (err <= 1.f) {
        c.accept = 1;
        c.t = c.last ? c.t_end : c.t + c.h;
        c.n_acc += 1;
        c.rho = c.rho_new;
        fac = 0.8f / cbrtf(ef);
        if (c.have_prev) fac = fac * ((float)c.h / (float)c.h_prev) * cbrtf(c.err_prev / ef);
        fac = fminf(fmaxf(fac, 0.1f), 10.f);
        if (c.after_reject && fac > 1.f) fac = 1.f;
        c.h_prev = c.h;
        c.err_prev = ef;
        c.have_prev = 1;
        c.after_reject = 0;
    } else {
        c.accept = 0;
        c.n_rej += 1;
        fac = fminf(fmaxf(0.8f / cbrtf(ef), 0.1f), 10.f);
        c.after_reject = 1;
    }
    c.h = (double)fac * c.h;
    rkc_plan(c, run, beta);
}

// ===========================================================================
// 2-D helpers shared by the single-CTA kernel (rkc.cu) and the cluster
// kernel (rkc_cl.cu).
// ===========================================================================
// ---------------------------------------------------------------------------
// FP32 right-hand side without time-step folding.
//   du = Du (G-1)^2, dv = Dv (G-1)^2;  FHN p2 = eps, p3 = a;  GM p2 = rho,
//   p3 = mu, deviation form with u0, v0, tu0 = 2 u0, e0 = u0 - mu v0,
//   e1 = u0^2 - v0;  BZ p2 = A, p3 = B, deviation form with u0 = A, v0 = B/A,
//   e0 = A (A v0 - B), c1 = 2 A v0 - (B+1), c2 = B - 2 A v0.
// ---------------------------------------------------------------------------
struct RkcK {
    float du, dv, p2, p3;
    float u0, v0, tu0, e0, e1, c1, c2;
};

inline RkcK make_rkc_k(const GroupDev &g) {
    RkcK k{};
    const double g2 = (double)(g.G - 1) * (double)(g.G - 1);
    k.du = (float)(g.p[0] * g2);
    k.dv = (float)(g.p[1] * g2);
    k.p2 = (float)g.p[2];
    k.p3 = (float)g.p[3];
    if (g.model == RD_GM) {
        const double mu = g.p[3];
        const float u0 = (float)(1.0 / mu);
        const float v0 = (float)((double)u0 * (double)u0);
        k.u0 = u0;
        k.v0 = v0;
        k.tu0 = 2.0f * u0;
        k.e0 = (float)((double)u0 - mu * (double)v0);
        k.e1 = (float)((double)u0 * (double)u0 - (double)v0);
    } else if (g.model == RD_BZ) {
        const double A = g.p[2], B = g.p[3];
        const float v0 = (float)(B / A);
        k.u0 = (float)A;
        k.v0 = v0;
        k.e0 = (float)(A * (A * (double)v0 - B));
        k.c1 = (float)(2.0 * A * (double)v0 - (B + 1.0));
        k.c2 = (float)(B - 2.0 * A * (double)v0);
    }
    return k;
}

// The RHS split for the stages: F_u = du Lu + ku Ru, F_v = dv Lv + kv Rv
// with the unscaled 5-point sums Lu, Lv and the kinetics' scale factors
// (ku, kv) = FHN (1, eps), GM (rho, rho), BZ (1, 1), DIFF (0, 0), so a
// stage folds du, dv, ku, kv into its per-stage weights.
template <int MODEL>
__device__ __forceinline__ void react_scale(const RkcK &k, float &ku, float &kv) {
    if (MODEL == RD_FHN) { ku = 1.f; kv = k.p2; }
    else if (MODEL == RD_GM) { ku = k.p2; kv = k.p2; }
    else if (MODEL == RD_BZ) { ku = 1.f; kv = 1.f; }
    else { ku = 0.f; kv = 0.f; }
}
template <int MODEL>
__device__ __forceinline__ void rhs_parts(float a, float b, const RkcK &k, float &Ru, float &Rv) {
    if (MODEL == RD_FHN) {
        Ru = fmaf(-a * a, a, a - b);
        Rv = fmaf(-k.p3, b, a);
    } else if (MODEL == RD_GM) {
        const float U = a + k.u0, V = b + k.v0;
        Ru = (U * fmaf(-k.p3, b, a + k.e0)) / V;
        Rv = fmaf(a, a + k.tu0, k.e1) - b;
    } else if (MODEL == RD_BZ) {
        const float U = a + k.u0;
        const float P = fmaf(k.v0 * a, a, (U * U) * b);
        Ru = fmaf(k.c1, a, k.e0 + P);
        Rv = fmaf(k.c2, a, -k.e0 - P);
    } else {
        Ru = 0.f;
        Rv = 0.f;
    }
}

// Gershgorin row sums of the Jacobian at one node (field values U, V; n =
// in-domain neighbours), the larger of the u and v rows.
template <int MODEL>
__device__ __forceinline__ float gersh_cell(float U, float V, float n, const RkcK &k) {
    float fu, fv, gu, gv;
    if (MODEL == RD_FHN) {
        fu = fmaf(-3.f * U, U, 1.f); fv = -1.f; gu = k.p2; gv = -k.p2 * k.p3;
    } else if (MODEL == RD_GM) {
        const float q = U / V;
        fu = k.p2 * fmaf(2.f, q, -k.p3); fv = -k.p2 * q * q; gu = 2.f * k.p2 * U; gv = -k.p2;
    } else if (MODEL == RD_BZ) {
        const float uv = U * V;
        fu = fmaf(2.f, uv, -(k.p3 + 1.f)); fv = U * U; gu = fmaf(-2.f, uv, k.p3); gv = -U * U;
    } else {
        fu = 0.f; fv = 0.f; gu = 0.f; gv = 0.f;
    }
    const float nu = n * k.du, nv = n * k.dv;
    const float ru = fabsf(fu - nu) + nu + fabsf(fv);
    const float rv = fabsf(gv - nv) + nv + fabsf(gu);
    return fmaxf(ru, rv);
}

// Kinetics increments R(Y_0 + d) - R(Y_0) in the unscaled form of
// rhs_parts (same scale factors ku, kv), exact in real arithmetic and formed
// from the increment (da, db), so their FP32 rounding is relative to the
// increment:
//   FHN: u^3 increment = da (u1^2 + u1 u0 + u0^2), u1 = a0 + da;
//   GM:  U^2 increment p = dU (2 U0 + dU),
//        U^2/V increment = (p V0 - U0^2 dV) / (V1 V0),  V1 = V0 + dV;
//   BZ:  U^2 V increment = p V1 + U0^2 dV.
template <int MODEL>
__device__ __forceinline__ void rhs_dparts(float a0, float b0, float da, float db, const RkcK &k, float &dRu,
                                           float &dRv) {
    if (MODEL == RD_FHN) {
        const float u1 = a0 + da;
        const float t = fmaf(u1, u1 + a0, a0 * a0);
        dRu = fmaf(-da, t, da - db);
        dRv = fmaf(-k.p3, db, da);
    } else if (MODEL == RD_GM) {
        const float U0 = a0 + k.u0, V0 = b0 + k.v0, V1 = V0 + db;
        const float p = da * fmaf(2.f, U0, da);
        const float q = __fdividef(fmaf(p, V0, -(U0 * U0) * db), V1 * V0);
        dRu = fmaf(-k.p3, da, q);
        dRv = p - db;
    } else if (MODEL == RD_BZ) {
        const float U0 = a0 + k.u0, V0 = b0 + k.v0, V1 = V0 + db;
        const float p = da * fmaf(2.f, U0, da);
        const float dP = fmaf(p, V1, (U0 * U0) * db);
        dRu = fmaf(-(k.p3 + 1.f), da, dP);
        dRv = fmaf(k.p3, da, -dP);
    } else {
        dRu = 0.f;
        dRv = 0.f;
    }
}

// Unscaled 5-point sum of an increment field: ((N + S) + (W + E)) - 4 d.
__device__ __forceinline__ float lap5(float d, float4 n) {
    return fmaf(-4.f, d, (n.x + n.y) + (n.z + n.w));
}

// Unscaled 5-point sum of the compensated state y + cy, with the rounding of
// the neighbour sum kept (TwoSum): ((N + S) + (W + E)) - 4 y is then exact
// (Sterbenz, the neighbours within a factor 2 of the node) up to the small
// error terms, to which the compensation's own sum is added.
__device__ __forceinline__ float lap5_exact(float y, float4 n, float lapc) {
    const float s1 = n.x + n.y, b1 = s1 - n.x, e1 = (n.x - (s1 - b1)) + (n.y - b1);
    const float s2 = n.z + n.w, b2 = s2 - n.z, e2 = (n.z - (s2 - b2)) + (n.w - b2);
    const float s3 = s1 + s2, b3 = s3 - s1, e3 = (s1 - (s3 - b3)) + (s2 - b3);
    return fmaf(-4.f, y, s3) + (((e1 + e2) + e3) + lapc);
}

// Block reduction of (sum of squares, max rho): warp shuffles, then warp 0
// combines the per-warp partials (every lane of warp 0 ends with the
// result).  red: 64 floats.
__device__ __forceinline__ void block_reduce2(float &ss, float &mx, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) { red[warp] = ss; red[32 + warp] = mx; }
    __syncthreads();
    if (warp == 0) {
        ss = lane < nw ? red[lane] : 0.f;
        mx = lane < nw ? red[32 + lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
    }
}

// G = 128: one realisation per thread-block cluster of 4 CTAs (rkc_cl.cu).
rd_status launch_rkc_cluster_group(const GroupDev &g, float *fields, const RkcRun &run, const float4 *tab,
                                   const double *beta, int64_t *stats, double *residual, uint32_t *status,
                                   cudaStream_t s);

}  // namespace rdcil
