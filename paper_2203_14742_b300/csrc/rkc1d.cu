// The 1-D reaction-diffusion-ODE model (Sec. 4.3, eq. rdode): its initial
// state and its adaptive stabilised second-order Runge-Kutta integration
// (App. B.2, the recurrence and step control of rkc.cu/rkc.cuh).
//
//   u_t = -u - u w + m1 q,   w_t = D w_xx - m3 w - u w + m2 q,
//   q = u^2 / (1 + k u^2),   params = (unused, D, m1, m2, m3, k),
// on G nodes, h = 1/(G-1), w_xx = ((w_{x+1} + w_{x-1}) - 2 w_x) (G-1)^2 with
// ghost = edge node; a realisation is [u, w][x].
//
// B300 design.  A realisation is small (2 x 64 values in the paper's
// setting), so one warp integrates one realisation: lane l holds nodes
// l*NPL .. l*NPL + NPL - 1 (NPL = G/32) of both species in registers, the
// w neighbours across lanes come from two shuffles per stage, and every
// lane runs an identical copy of the step control on butterfly-reduced
// values, so the kernel has no barrier and no shared memory at all.
#include <cmath>
#include "common.cuh"
#include "rkc.cuh"

namespace rdcil {

// ---------------------------------------------------------------------------
// Initial state: u = U(lo, hi) noise smoothed by RD_RDODE_SMOOTH passes of
// ((u_{x-1} + u_x) + u_{x+1}) / 3 (ghost = edge node), FP64 with every
// operation rounded separately, rounded once to FP32; w = 0.
// ---------------------------------------------------------------------------
template <int NPL>
__global__ void __launch_bounds__(128) rdode_init_kernel(float *__restrict__ fields, int64_t field_offset,
                                                         int n_real, uint64_t seed, double lo, double hi) {
    constexpr int N = 32 * NPL;
    const int wid = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= n_real) return;
    const double span = __dsub_rn(hi, lo);
    double a[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int x = lane * NPL + i;
        const uint64_t z = splitmix64_at(seed, (uint64_t)wid * 2u * (uint64_t)N + (uint64_t)x);
        const double U = (double)(z >> 11) * 0x1.0p-53;
        a[i] = __dadd_rn(lo, __dmul_rn(span, U));
    }
    for (int it = 0; it < RD_RDODE_SMOOTH; ++it) {
        double l0 = __shfl_up_sync(0xffffffffu, a[NPL - 1], 1);
        double r0 = __shfl_down_sync(0xffffffffu, a[0], 1);
        if (lane == 0) l0 = a[0];
        if (lane == 31) r0 = a[NPL - 1];
        double b[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const double l = i > 0 ? a[i - 1] : l0, r = i < NPL - 1 ? a[i + 1] : r0;
            b[i] = __ddiv_rn(__dadd_rn(__dadd_rn(l, a[i]), r), 3.0);
        }
#pragma unroll
        for (int i = 0; i < NPL; ++i) a[i] = b[i];
    }
    float *base = fields + field_offset + (int64_t)wid * 2 * N;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        base[lane * NPL + i] = __double2float_rn(a[i]);
        base[N + lane * NPL + i] = 0.0f;
    }
}

rd_status launch_rdode_init(const GroupDev &g, float *fields, cudaStream_t s) {
    const unsigned grid = (unsigned)((g.n_real + 3) / 4);
    switch (g.G) {
        case 32: rdode_init_kernel<1><<<grid, 128, 0, s>>>(fields, g.field_offset, g.n_real, g.seed, g.noise_lo, g.noise_hi); break;
        case 64: rdode_init_kernel<2><<<grid, 128, 0, s>>>(fields, g.field_offset, g.n_real, g.seed, g.noise_lo, g.noise_hi); break;
        case 128: rdode_init_kernel<4><<<grid, 128, 0, s>>>(fields, g.field_offset, g.n_real, g.seed, g.noise_lo, g.noise_hi); break;
        case 256: rdode_init_kernel<8><<<grid, 128, 0, s>>>(fields, g.field_offset, g.n_real, g.seed, g.noise_lo, g.noise_hi); break;
        default: return RD_ERR_UNSUPPORTED;
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Adaptive integration, one warp per realisation.
// ---------------------------------------------------------------------------
struct Rkc1K {
    float dd;                 // D (G-1)^2
    float m1, m2, m3, k;
};

// Butterfly reductions: every lane ends with the same value.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// w neighbours of every node of the lane (ghost = edge node at the ends).
template <int NPL>
__device__ __forceinline__ void w_neighbours(const float (&w)[NPL], int lane, float (&wl)[NPL], float (&wr)[NPL]) {
    float l0 = __shfl_up_sync(0xffffffffu, w[NPL - 1], 1);
    float r0 = __shfl_down_sync(0xffffffffu, w[0], 1);
    if (lane == 0) l0 = w[0];
    if (lane == 31) r0 = w[NPL - 1];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        wl[i] = i > 0 ? w[i - 1] : l0;
        wr[i] = i < NPL - 1 ? w[i + 1] : r0;
    }
}

// Kinetics: R_u = -u - u w + m1 q,  R_w = -m3 w - u w + m2 q.  (The
// quotients here and below use the 2-ulp fast division: they sit on the
// latency chain of a warp's stage, and FP32 state rounding dominates.)
__device__ __forceinline__ void kin1(float u, float w, const Rkc1K &K, float &Ru, float &Rw) {
    const float uu = u * u;
    const float q = __fdividef(uu, fmaf(K.k, uu, 1.f));
    Ru = fmaf(K.m1, q, fmaf(-u, w, -u));
    Rw = fmaf(K.m2, q, fmaf(-u, w, -K.m3 * w));
}

// Kinetics increments R(Y_0 + d) - R(Y_0), exact in real arithmetic and
// formed from the increment itself, so their FP32 rounding is relative to
// the (small) increment rather than to R:
//   q(u0 + du) - q(u0) = du (2 u0 + du) / ((1 + k u1^2)(1 + k u0^2)),  u1 = u0 + du,
//   -(u w) increment = -(u0 dw + du w1),  w1 = w0 + dw.
__device__ __forceinline__ void dkin1(float u0, float w0, float du, float dw, const Rkc1K &K, float &dRu,
                                      float &dRw) {
    const float u1 = u0 + du, w1 = w0 + dw;
    const float den0 = fmaf(K.k, u0 * u0, 1.f), den1 = fmaf(K.k, u1 * u1, 1.f);
    const float dq = __fdividef(du * fmaf(2.f, u0, du), den0 * den1);
    const float t = fmaf(u0, dw, du * w1);
    dRu = fmaf(K.m1, dq, -du - t);
    dRw = fmaf(K.m2, dq, fmaf(-K.m3, dw, -t));
}

// Gershgorin row sums at one node with n in-domain neighbours.
__device__ __forceinline__ float gersh1(float u, float w, float n, const Rkc1K &K) {
    const float den = fmaf(K.k, u * u, 1.f);
    const float dq = __fdividef(2.f * u, den * den);
    const float fu = fmaf(K.m1, dq, -1.f - w), fw = -u;
    const float gu = fmaf(K.m2, dq, -w), gw = -K.m3 - u;
    const float nd = n * K.dd;
    return fmaxf(fabsf(fu) + fabsf(fw), fabsf(gw - nd) + nd + fabsf(gu));
}

template <int NPL>
__global__ void __launch_bounds__(128) rd_rkc1d_kernel(float *__restrict__ fields, int64_t field_offset, int n_real,
                                                       Rkc1K K, RkcRun run, double t_end,
                                                       const float4 *__restrict__ tab, const double *__restrict__ beta,
                                                       int64_t *__restrict__ stats, double D, double m1, double m2,
                                                       double m3, double kk, double *__restrict__ residual,
                                                       uint32_t *__restrict__ status) {
    constexpr int N = 32 * NPL;
    // beta(s) in shared memory for the stage-count search on each warp's
    // serial control path (loaded before any warp leaves)
    __shared__ double betaS[RKC_STRIDE];
    for (int i = threadIdx.x; i < RKC_STRIDE; i += blockDim.x) betaS[i] = beta[i];
    __syncthreads();
    const int wid = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= n_real) return;                       // whole warps only
    float *base = fields + field_offset + (int64_t)wid * 2 * N;
    const bool adaptive = run.s_fixed < 2;
    // Every RHS evaluation of a step is written as F(Y_0 + D) = F_0 + dF with
    // F_0 = F(Y_0) evaluated once from the stored state and
    //   dF_u = dR_u,  dF_w = dd Lap(D_w) + dR_w
    // formed from the increment D (dkin1), which is the same method in real
    // arithmetic.  The FP32 rounding of F_0 (from the large Laplacian and
    // kinetics terms) is then common to every evaluation of the step and
    // cancels exactly in the error estimate, whose stage weights sum to one,
    // and the rounding of each evaluation is relative to the increment.
    // The diffusing species is held compensated, w = y0w + c0w (c0w the
    // exact FP32 rounding residuals of the accepted updates, TwoSum): an
    // FP32 state alone cannot sit at the discrete equilibrium, so every
    // step would leave stiff diffusion modes of amplitude ~ulp(w)/2, and the
    // error estimate reports about 0.4 |h lambda| times such a mode (it is
    // not an estimate of the stiff modes' true local error), which would
    // hold h lambda_max near tol / ulp.  u does not diffuse and needs no
    // compensation.
    float y0u[NPL], y0w[NPL], c0w[NPL], f0u[NPL], f0w[NPL], d1u[NPL], d1w[NPL], d2u[NPL], d2w[NPL];
    float yu[NPL], yw[NPL], fsu[NPL], fsw[NPL];
    float nb[NPL];                                   // in-domain neighbour count
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int x = lane * NPL + i;
        y0u[i] = base[x];
        y0w[i] = base[N + x];
        c0w[i] = 0.f;
        nb[i] = (float)((x > 0) + (x < N - 1));
    }
    // F(Y_0) from the stored state; rho(Y_0)
    // (the Laplacian of the compensated w, Lap(y0w) + Lap(c0w), with the
    // neighbour sum's rounding error kept: its rounding, times D (G-1)^2,
    // would otherwise change F_0 by ~ulp(w) D (G-1)^2 from step to step and
    // shift the stiff modes' equilibrium by ulp-sized amounts)
    auto eval0 = [&](float &rmax) {
        float wl[NPL], wr[NPL], cl[NPL], cr[NPL];
        w_neighbours<NPL>(y0w, lane, wl, wr);
        w_neighbours<NPL>(c0w, lane, cl, cr);
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            float Ru, Rw;
            kin1(y0u[i], y0w[i], K, Ru, Rw);
            f0u[i] = Ru;
            // (wl + wr) by TwoSum; (wl + wr) - 2 w is then exact (Sterbenz,
            // neighbours within a factor 2) up to the small error terms
            const float s1 = wl[i] + wr[i];
            const float bp = s1 - wl[i];
            const float e1 = (wl[i] - (s1 - bp)) + (wr[i] - bp);
            const float L = fmaf(-2.f, y0w[i], s1) + (e1 + fmaf(-2.f, c0w[i], cl[i] + cr[i]));
            f0w[i] = fmaf(K.dd, L, Rw);
            if (adaptive) rmax = fmaxf(rmax, gersh1(y0u[i], y0w[i], nb[i], K));
        }
    };
    float rmax = 0.f;
    eval0(rmax);
    RkcCtl c;
    c.t = 0.0;
    c.t_end = t_end;
    c.h = run.h0;
    c.h_prev = 0.0;
    c.err_prev = 0.f;
    c.attempts = 0;
    c.n_acc = 0;
    c.n_rej = 0;
    c.n_rhs = 1;
    c.rho = warp_max(rmax);
    c.s = 0;
    c.s_used = 0;
    c.have_prev = 0;
    c.after_reject = 0;
    c.accept = 0;
    c.done = 0;
    c.fail = 0;
    rkc_plan(c, run, betaS);

    // one stage j >= 2: dp <- mu dl + nu dp + mt h F(Y_0 + dl) + gt h F_0
    //                       = mu dl + nu dp + (mt + gt) h F_0 + mt h dF(dl)
    auto stage = [&](const float (&dlu)[NPL], const float (&dlw)[NPL], float (&dpu)[NPL], float (&dpw)[NPL],
                     const float4 cj, float h) {
        const float mth = cj.z * h, cfh = (cj.z + cj.w) * h, mdd = mth * K.dd;
        float dl[NPL], dr[NPL];
        w_neighbours<NPL>(dlw, lane, dl, dr);
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            float dRu, dRw;
            dkin1(y0u[i], y0w[i], dlu[i], dlw[i], K, dRu, dRw);
            const float L = fmaf(-2.f, dlw[i], dl[i] + dr[i]);
            dpu[i] = fmaf(cj.x, dlu[i], fmaf(cj.y, dpu[i], fmaf(mth, dRu, cfh * f0u[i])));
            dpw[i] = fmaf(cj.x, dlw[i], fmaf(cj.y, dpw[i], fmaf(mdd, L, fmaf(mth, dRw, cfh * f0w[i]))));
        }
    };

    while (!c.done) {
        const int s = c.s;
        const float h = c.hf;
        const float4 *row = tab + (size_t)s * RKC_STRIDE;
        const float m1h = __ldg(&row[1].z) * h;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            d1u[i] = m1h * f0u[i];
            d1w[i] = m1h * f0w[i];
            d2u[i] = 0.f;
            d2w[i] = 0.f;
        }
        float4 cn = __ldg(&row[2]);
        for (int j = 2; j <= s; j += 2) {
            const float4 cj = cn;
            cn = __ldg(&row[j + 1 <= s ? j + 1 : s]);
            stage(d1u, d1w, d2u, d2w, cj, h);
            if (j + 1 > s) {
#pragma unroll
                for (int i = 0; i < NPL; ++i) { d1u[i] = d2u[i]; d1w[i] = d2w[i]; }
                break;
            }
            const float4 ck = cn;
            cn = __ldg(&row[j + 2 <= s ? j + 2 : s]);
            stage(d2u, d2w, d1u, d1w, ck, h);
        }
        // Y_s, F(Y_s), error estimate, rho(Y_s)
        float acc = 0.f;
        rmax = 0.f;
        {
            const float rtol = (float)run.rtol, atol = (float)run.atol, h04 = 0.4f * h;
            float dl[NPL], dr[NPL];
            w_neighbours<NPL>(d1w, lane, dl, dr);
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                yu[i] = y0u[i] + d1u[i];
                yw[i] = y0w[i] + d1w[i];
                // dF(D_s) = F(Y_s) - F_0
                float dRu, dRw;
                dkin1(y0u[i], y0w[i], d1u[i], d1w[i], K, dRu, dRw);
                fsu[i] = dRu;
                fsw[i] = fmaf(K.dd, fmaf(-2.f, d1w[i], dl[i] + dr[i]), dRw);
                if (adaptive) {
                    // est = (12 (Y_0 - Y_s) + 6 h (F_0 + F_s)) / 15
                    //     = -0.8 D_s + 0.4 h (2 F_0 + dF(D_s))
                    const float eu = fmaf(-0.8f, d1u[i], h04 * fmaf(2.f, f0u[i], fsu[i]));
                    const float ew = fmaf(-0.8f, d1w[i], h04 * fmaf(2.f, f0w[i], fsw[i]));
                    const float qu = __fdividef(eu, fmaf(rtol, fmaxf(fabsf(y0u[i]), fabsf(yu[i])), atol));
                    const float qw = __fdividef(ew, fmaf(rtol, fmaxf(fabsf(y0w[i]), fabsf(yw[i])), atol));
                    acc = fmaf(qu, qu, fmaf(qw, qw, acc));
                    rmax = fmaxf(rmax, gersh1(yu[i], yw[i], nb[i], K));
                }
            }
        }
        const float ss = warp_sum(acc);
        c.rho_new = warp_max(rmax);
        rkc_decide(c, run, betaS, ss, 2 * N);
        if (c.accept) {
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                y0u[i] = yu[i];
                // (y0w + c0w) + D_s, compensated: TwoSum of y0w and D_s,
                // the error added to c0w, renormalised
                const float sw = y0w[i] + d1w[i];
                const float bp = sw - y0w[i];
                const float e = (y0w[i] - (sw - bp)) + (d1w[i] - bp);
                const float lo = c0w[i] + e;
                y0w[i] = sw + lo;
                c0w[i] = lo - (y0w[i] - sw);
            }
            // F(Y_0) afresh from the stored (rounded) state, not
            // F_0 + dF(D_s), so the run keeps solving the discrete system
            // of the state it holds
            float dummy = 0.f;
            if (!c.done) eval0(dummy);
        }
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        base[lane * NPL + i] = y0u[i];
        base[N + lane * NPL + i] = y0w[i];
    }
    if (lane == 0) {
        if (stats) {
            int64_t *st = stats + 4 * (int64_t)wid;
            st[0] = c.n_acc;
            st[1] = c.n_rej;
            st[2] = c.n_rhs;
            st[3] = c.s_used;
        }
        if (c.fail == 1) atomicOr(status, (unsigned)ST_STEPFAIL);
        if (c.fail == 2) atomicOr(status, (unsigned)ST_NONFINITE);
    }
    // FP64 steady-state residual of the final FP32 state (the plain
    // operation order of the definition, every operation rounded)
    {
        const double g2 = (double)(N - 1) * (double)(N - 1);
        double mx = 0.0, sq = 0.0;
        bool bad = false;
        double wv[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) wv[i] = (double)y0w[i];
        double l0 = __shfl_up_sync(0xffffffffu, wv[NPL - 1], 1);
        double r0 = __shfl_down_sync(0xffffffffu, wv[0], 1);
        if (lane == 0) l0 = wv[0];
        if (lane == 31) r0 = wv[NPL - 1];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const double u = (double)y0u[i], w = wv[i];
            const double wl = i > 0 ? wv[i - 1] : l0, wr = i < NPL - 1 ? wv[i + 1] : r0;
            const double lap = __dmul_rn(__dsub_rn(__dadd_rn(wr, wl), __dmul_rn(2.0, w)), g2);
            const double uu = __dmul_rn(u, u);
            const double q = __ddiv_rn(uu, __dadd_rn(1.0, __dmul_rn(kk, uu)));
            const double uv = __dmul_rn(u, w);
            const double Fu = __dadd_rn(__dsub_rn(-u, uv), __dmul_rn(m1, q));
            const double Fw = __dadd_rn(__dmul_rn(D, lap),
                                        __dadd_rn(__dsub_rn(-__dmul_rn(m3, w), uv), __dmul_rn(m2, q)));
            bad |= !isfinite(u) || !isfinite(w) || !isfinite(Fu) || !isfinite(Fw);
            mx = fmax(mx, fmax(fabs(Fu), fabs(Fw)));
            sq = __dadd_rn(sq, __dadd_rn(__dmul_rn(Fu, Fu), __dmul_rn(Fw, Fw)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
        }
        const bool anybad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            if (anybad) {
                atomicOr(status, (unsigned)ST_NONFINITE);
                mx = __longlong_as_double(0x7ff8000000000000ll);
                sq = mx;
            }
            if (residual) {
                residual[2 * wid] = mx;
                residual[2 * wid + 1] = sqrt(sq / (double)(2 * N));
            }
        }
    }
}

bool rkc1d_supported(const GroupDev &g) {
    return g.model == RD_RDODE && (g.G == 32 || g.G == 64 || g.G == 128 || g.G == 256);
}

rd_status launch_rkc1d_group(const GroupDev &g, const float4 *tab, const double *beta, float *fields,
                             const rd_rkc_opts &o, int64_t *stats, double *residual, uint32_t *status,
                             cudaStream_t s) {
    RkcRun run{o.t_end, o.h0, o.rtol, o.atol, o.s_max, o.s_fixed, o.n_fixed, o.max_attempts};
    const double g2 = (double)(g.G - 1) * (double)(g.G - 1);
    Rkc1K K{(float)(g.p[1] * g2), (float)g.p[2], (float)g.p[3], (float)g.p[4], (float)g.p[5]};
    const double t_end = o.t_end > 0.0 ? o.t_end : g.dt * (double)g.n_steps;
    int64_t *st_g = stats ? stats + 4 * g.real_base : nullptr;
    double *res_g = residual ? residual + 2 * g.real_base : nullptr;
    const unsigned grid = (unsigned)((g.n_real + 3) / 4);
#define RKC1D_LAUNCH(NPL)                                                                                        \
    rd_rkc1d_kernel<NPL><<<grid, 128, 0, s>>>(fields, g.field_offset, g.n_real, K, run, t_end, tab, beta, st_g, \
                                              g.p[1], g.p[2], g.p[3], g.p[4], g.p[5], res_g, status)
    switch (g.G) {
        case 32: RKC1D_LAUNCH(1); break;
        case 64: RKC1D_LAUNCH(2); break;
        case 128: RKC1D_LAUNCH(4); break;
        case 256: RKC1D_LAUNCH(8); break;
        default: return RD_ERR_UNSUPPORTED;
    }
#undef RKC1D_LAUNCH
    note_launch();
    return cuda_status(cudaGetLastError());
}

}  // namespace rdcil
