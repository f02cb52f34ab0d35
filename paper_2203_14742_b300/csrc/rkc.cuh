// Step control of the stabilised second-order Runge-Kutta integrator
// (App. B.2), shared by the 2-D kernel (rkc.cu, thread 0 of a CTA owns the
// state in shared memory) and the 1-D kernel (rkc1d.cu, every lane of a
// warp holds an identical copy in registers).  Coefficient tables:
// rkc_tables() builds, once per process, tab[s][j] = (mu_j, nu_j, mt_j,
// gt_j) (FP32, s = 2..RD_RKC_S_MAX, j = 1..s) and beta[s] (FP64).
#pragma once
#include "common.cuh"

namespace rdcil {

constexpr int RKC_SMAX = RD_RKC_S_MAX;
constexpr int RKC_STRIDE = RKC_SMAX + 1;

rd_status rkc_tables(cudaStream_t s, const float4 **tab, const double **beta);

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

}  // namespace rdcil
