// Stabilised explicit second-order Runge-Kutta integration of the batched
// reaction-diffusion systems (App. B.2): stages by a three-term recurrence,
// stage number from a Gershgorin bound of the Jacobian's spectral radius,
// weighted RMS error estimate and a predictive step-size controller
// (eta = 0.8), all on the GPU.  The coefficients are those of the
// second-order Runge-Kutta-Chebyshev method (damping eps = 2/13), the member
// of the family with closed-form coefficients, since the paper does not
// print ROCK2's:
//   w0 = 1 + eps/s^2,  w1 = T_s'(w0)/T_s''(w0),  b_j = T_j''(w0)/T_j'(w0)^2
//   (b_0 = b_1 = b_2),  a_j = 1 - b_j T_j(w0),
//   Y_1 = Y_0 + mt_1 h F(Y_0),  mt_1 = b_1 w1,
//   Y_j = (1-mu_j-nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2} + mt_j h F(Y_{j-1}) + gt_j h F(Y_0),
//   mu_j = 2 b_j w0/b_{j-1}, nu_j = -b_j/b_{j-2}, mt_j = 2 b_j w1/b_{j-1}, gt_j = -a_{j-1} mt_j,
//   stable for h rho <= beta(s) = (1 + w0)/w1.
//
// B300 design.  One CTA integrates one realisation for its whole adaptive
// run, with no host round trip: the state lives in register tiles (the
// natural-order tiles of tile.cuh), each stage is one halo exchange
// through the shared-memory ring and one barrier, and thread 0 takes the
// step-control decisions in FP64 from block reductions.  (The paper's GPU
// solver kept the vectors in global memory and synchronised with the host
// after every stage.)
//
// Precision.  The recurrence is carried on the increments D_j = Y_j - Y_0,
//   D_1 = mt_1 h F_0,  D_j = mu_j D_{j-1} + nu_j D_{j-2} + mt_j h F(Y_0 + D_{j-1}) + gt_j h F_0,
// which is the same recurrence (the stage weights sum to one), so the FP32
// rounding of the stages is relative to the small increments rather than to
// the state (with the plain form, mu_j ~ 2 and nu_j ~ -1 amplify the
// state's rounding through the stages).  GM and BZ states are kept as the
// deviation from the FP32 equilibrium, as in the Euler stepper.  The error
// estimate uses Y_0 - Y_s = -D_s, free of cancellation.
#include <cmath>
#include <cstdio>
#include <mutex>
#include "common.cuh"
#include "tile.cuh"
#include "rkc.cuh"

namespace rdcil {


// ---------------------------------------------------------------------------
// Coefficient table: tab[s][j] = (mu_j, nu_j, mt_j, gt_j) in FP32 for
// s = 2..RKC_SMAX, j = 1..s; beta[s] in FP64.  One thread per s.
// ---------------------------------------------------------------------------
__global__ void rkc_table_kernel(float4 *__restrict__ tab, double *__restrict__ beta) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < 2 || s > RKC_SMAX) return;
    const double w0 = 1.0 + (2.0 / 13.0) / ((double)s * (double)s);
    // first pass: T_s', T_s'' at w0 -> w1
    double T0 = 1.0, T1v = w0, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
    for (int j = 2; j <= s; ++j) {
        const double T2v = 2.0 * w0 * T1v - T0;
        const double d2 = 2.0 * T1v + 2.0 * w0 * d1 - d0;
        const double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
        T0 = T1v; T1v = T2v; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
    }
    const double w1 = d1 / e1;
    beta[s] = (1.0 + w0) / w1;
    // second pass: b_j, a_j and the stage coefficients
    T0 = 1.0; T1v = w0; d0 = 0.0; d1 = 1.0; e0 = 0.0; e1 = 0.0;
    // b_2 = T_2''/T_2'^2 = 4 / (4 w0)^2 first (b_0 = b_1 = b_2)
    const double b2 = 4.0 / ((4.0 * w0) * (4.0 * w0));
    double bjm2 = b2, bjm1 = b2;                 // b_{j-2}, b_{j-1}
    double ajm1 = 1.0 - b2 * w0;                 // a_1
    float4 *row = tab + (size_t)s * RKC_STRIDE;
    row[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    row[1] = make_float4(0.f, 0.f, (float)(b2 * w1), 0.f);
    for (int j = 2; j <= s; ++j) {
        const double T2v = 2.0 * w0 * T1v - T0;
        const double d2 = 2.0 * T1v + 2.0 * w0 * d1 - d0;
        const double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
        const double bj = e2 / (d2 * d2);
        const double mu = 2.0 * bj * w0 / bjm1;
        const double nu = -bj / bjm2;
        const double mt = 2.0 * bj * w1 / bjm1;
        const double gt = -ajm1 * mt;
        row[j] = make_float4((float)mu, (float)nu, (float)mt, (float)gt);
        ajm1 = 1.0 - bj * T2v;
        bjm2 = bjm1;
        bjm1 = bj;
        T0 = T1v; T1v = T2v; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
    }
}

// bytes of the coefficient table followed by the beta table (one
// allocation of the handle; the beta part starts 16-byte aligned)
size_t rkc_table_bytes() {
    return sizeof(float4) * (size_t)RKC_STRIDE * RKC_STRIDE + sizeof(double) * RKC_STRIDE;
}

rd_status rkc_tables_fill(float4 *tab, double *beta, cudaStream_t s) {
    RD_CUDA_TRY(cudaMemsetAsync(beta, 0, sizeof(double) * RKC_STRIDE, s));
    rkc_table_kernel<<<(RKC_STRIDE + 127) / 128, 128, 0, s>>>(tab, beta);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// Exchange the edge rows of a tile quantity (yu, yv) through ring buffer hb
// (one barrier); tile_apply then calls body(i, c, nu, nv) with the four
// neighbours (N, S, W, E) of every node as float4 (mirror ghosts at the
// domain edge).
template <int G, int TY, int TX>
__device__ __forceinline__ void tile_exchange(float *hb, int tx, int ty, const float (&yu)[TY][TX],
                                              const float (&yv)[TY][TX]) {
    halo_put<G, TY, TX>(hb, tx, ty, yu, yv);
    __syncthreads();
}

template <int G, int TY, int TX, class Body>
__device__ __forceinline__ void tile_apply(const float *hb, int tx, int ty, const float (&yu)[TY][TX],
                                           const float (&yv)[TY][TX], Body body) {
    constexpr int NX = Tiling<G, TY, TX>::NX;
    float pu[TX], pv[TX];
    halo_north<G, TY, TX>(hb, tx, ty, yu, yv, pu, pv);
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        float su[TX], sv[TX];
        row_south<G, TY, TX>(hb, tx, ty, i, yu, yv, su, sv);
        float wu, eu, wv, ev;
        row_west_east<NX>(tx, yu[i][0], yu[i][TX - 1], wu, eu);
        row_west_east<NX>(tx, yv[i][0], yv[i][TX - 1], wv, ev);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            const float Lu = c > 0 ? yu[i][c - 1] : wu, Ru = c < TX - 1 ? yu[i][c + 1] : eu;
            const float Lv = c > 0 ? yv[i][c - 1] : wv, Rv = c < TX - 1 ? yv[i][c + 1] : ev;
            body(i, c, make_float4(pu[c], su[c], Lu, Ru), make_float4(pv[c], sv[c], Lv, Rv));
        }
#pragma unroll
        for (int c = 0; c < TX; ++c) { pu[c] = yu[i][c]; pv[c] = yv[i][c]; }
    }
}

// One stage j >= 2 in increment form: with F(Y_0 + D) = F_0 + dF(D),
//   dF_u(D) = du Lap(D_u) + ku dR_u(Y_0; D)   (likewise v),
//   D_j = mu_j D_{j-1} + nu_j D_{j-2} + (mt_j + gt_j) h F_0 + mt_j h dF(D_{j-1}),
// the same recurrence as the stage form in real arithmetic.  D_{j-1} (dl)
// is exchanged; D_j is written over D_{j-2} (dp).  Coefficients from
// crow[j] (shared memory, read after the exchange barrier).
template <int MODEL, int G, int TY, int TX>
__device__ __forceinline__ void rkc_stage(float *hb, int tx, int ty, const float (&y0u)[TY][TX],
                                          const float (&y0v)[TY][TX], const float (&f0u)[TY][TX],
                                          const float (&f0v)[TY][TX], const float (&dlu)[TY][TX],
                                          const float (&dlv)[TY][TX], float (&dpu)[TY][TX], float (&dpv)[TY][TX],
                                          const float4 *crow, int j, float h, const RkcK &k) {
    tile_exchange<G, TY, TX>(hb, tx, ty, dlu, dlv);
    const float4 cj = crow[j];
    const float mth = cj.z * h, cfh = (cj.z + cj.w) * h;
    float ku, kv;
    react_scale<MODEL>(k, ku, kv);
    const float mdu = mth * k.du, mdv = mth * k.dv, mru = mth * ku, mrv = mth * kv;
    tile_apply<G, TY, TX>(hb, tx, ty, dlu, dlv, [&](int i, int c, float4 nu, float4 nv) {
        float gu = cfh * f0u[i][c], gv = cfh * f0v[i][c];
        if (MODEL != RD_DIFF) {
            float dRu, dRv;
            rhs_dparts<MODEL>(y0u[i][c], y0v[i][c], dlu[i][c], dlv[i][c], k, dRu, dRv);
            gu = fmaf(mru, dRu, gu);
            gv = fmaf(mrv, dRv, gv);
        }
        dpu[i][c] = fmaf(cj.x, dlu[i][c], fmaf(cj.y, dpu[i][c], fmaf(mdu, lap5(dlu[i][c], nu), gu)));
        dpv[i][c] = fmaf(cj.x, dlv[i][c], fmaf(cj.y, dpv[i][c], fmaf(mdv, lap5(dlv[i][c], nv), gv)));
    });
}

// Shared memory (byte offsets): halo ring at 0 | 64 doubles of reduction
// scratch | RkcCtl | coefficient row float4[RKC_STRIDE] at a 16-byte
// boundary | beta[RKC_STRIDE] doubles | the state's compensation
// [species 2][G][G] floats at a 16-byte boundary.
template <int G, int TY, int TX>
__host__ __device__ constexpr size_t rkc_red_off() {
    return Tiling<G, TY, TX>::SMEM;
}
template <int G, int TY, int TX>
__host__ __device__ constexpr size_t rkc_ctl_off() {
    return rkc_red_off<G, TY, TX>() + 64 * sizeof(double);
}
template <int G, int TY, int TX>
__host__ __device__ constexpr size_t rkc_crow_off() {
    return (rkc_ctl_off<G, TY, TX>() + sizeof(RkcCtl) + 15) / 16 * 16;
}
template <int G, int TY, int TX>
__host__ __device__ constexpr size_t rkc_beta_off() {
    return rkc_crow_off<G, TY, TX>() + RKC_STRIDE * sizeof(float4);
}
template <int G, int TY, int TX>
__host__ __device__ constexpr size_t rkc_c0_off() {
    return (rkc_beta_off<G, TY, TX>() + RKC_STRIDE * sizeof(double) + 15) / 16 * 16;
}
template <int G, int TY, int TX>
__host__ __device__ constexpr size_t rkc_smem() {
    return rkc_c0_off<G, TY, TX>() + 2 * (size_t)G * G * sizeof(float);
}

template <int MODEL, int G, int TY, int TX>
__global__ void __launch_bounds__(Tiling<G, TY, TX>::NT, 1)
rd_rkc_kernel(float *__restrict__ fields, int64_t field_offset, RkcK k, RkcRun run, double t_end,
              const float4 *__restrict__ tab, const double *__restrict__ beta, int64_t *__restrict__ stats,
              double p0, double p1, double p2, double p3, double *__restrict__ residual,
              uint32_t *__restrict__ status) {
    using T = Tiling<G, TY, TX>;
    constexpr int NX = T::NX;
    constexpr int M = 2 * G * G;
    extern __shared__ float4 smem_f4[];
    static_assert(rkc_red_off<G, TY, TX>() % 16 == 0 && rkc_ctl_off<G, TY, TX>() % 16 == 0 &&
                      rkc_crow_off<G, TY, TX>() % 16 == 0 && rkc_beta_off<G, TY, TX>() % 16 == 0 &&
                      rkc_c0_off<G, TY, TX>() % 16 == 0,
                  "shared-memory regions must start on 16-byte boundaries");
    char *sb = reinterpret_cast<char *>(smem_f4);
    float *ring = reinterpret_cast<float *>(sb);
    double *red = reinterpret_cast<double *>(sb + rkc_red_off<G, TY, TX>());
    RkcCtl &c = *reinterpret_cast<RkcCtl *>(sb + rkc_ctl_off<G, TY, TX>());
    float4 *crow = reinterpret_cast<float4 *>(sb + rkc_crow_off<G, TY, TX>());
    double *betaS = reinterpret_cast<double *>(sb + rkc_beta_off<G, TY, TX>());
    // The state is held compensated: node value = y0 (registers) + c0
    // (shared memory), c0 the exact FP32 rounding residuals of the accepted
    // updates (TwoSum).  An FP32 state alone cannot sit at the discrete
    // equilibrium, so each step would leave stiff diffusion modes of
    // amplitude ~ulp/2, and the error estimate reports about 0.4 |h lambda|
    // times such a mode (it does not estimate the stiff modes' true local
    // error), which would hold h lambda_max near tol / ulp.
    float *c0 = reinterpret_cast<float *>(sb + rkc_c0_off<G, TY, TX>());
    const int tid = threadIdx.x, tx = tid % NX, ty = tid / NX;
    for (int i = tid; i < RKC_STRIDE; i += blockDim.x) betaS[i] = beta[i];
    const int r = blockIdx.x;
    float *base = fields + field_offset + (int64_t)r * M;
    const bool adaptive = run.s_fixed < 2;
    float ku, kv;
    react_scale<MODEL>(k, ku, kv);

    float y0u[TY][TX], y0v[TY][TX], f0u[TY][TX], f0v[TY][TX];
    float d1u[TY][TX], d1v[TY][TX], d2u[TY][TX], d2v[TY][TX];
    tile_load<G, TY, TX>(base, tx, ty, y0u, y0v);
    {
        CoefF cf{};
        cf.u0 = k.u0;
        cf.v0 = k.v0;
        tile_to_state<MODEL, TY, TX>(y0u, y0v, cf);
    }
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int cc = 0; cc < TX; ++cc) {
            const int node = (ty * TY + i) * G + tx * TX + cc;
            c0[node] = 0.f;
            c0[G * G + node] = 0.f;
        }
    // in-domain neighbour count of each node (Gershgorin row weights)
    auto ncount = [&](int i, int cc) {
        const int y = ty * TY + i, x = tx * TX + cc;
        return (float)((x > 0) + (x < G - 1) + (y > 0) + (y < G - 1));
    };
    // 5-point sum of the compensation at node (y, x) of species sp
    auto lapc = [&](int sp, int y, int x) {
        const float *cs = c0 + sp * G * G;
        const float ce = cs[y * G + x];
        const float n = cs[(y > 0 ? y - 1 : y) * G + x], so = cs[(y < G - 1 ? y + 1 : y) * G + x];
        const float w = cs[y * G + (x > 0 ? x - 1 : x)], e = cs[y * G + (x < G - 1 ? x + 1 : x)];
        return fmaf(-4.f, ce, (n + so) + (w + e));
    };

    int hk = 0;
    // F_0 = F(Y_0) of the stored compensated state (the kinetics at y0; the
    // compensation, below ulp/2, only enters the stiff diffusion term)
    auto eval0 = [&]() {
        tile_exchange<G, TY, TX>(ring + hk * (T::HALO_FLOATS / 2), tx, ty, y0u, y0v);
        tile_apply<G, TY, TX>(ring + hk * (T::HALO_FLOATS / 2), tx, ty, y0u, y0v,
                              [&](int i, int cc, float4 nu, float4 nv) {
                                  const int y = ty * TY + i, x = tx * TX + cc;
                                  const float Lu = lap5_exact(y0u[i][cc], nu, lapc(0, y, x));
                                  const float Lv = lap5_exact(y0v[i][cc], nv, lapc(1, y, x));
                                  float Ru, Rv;
                                  rhs_parts<MODEL>(y0u[i][cc], y0v[i][cc], k, Ru, Rv);
                                  f0u[i][cc] = fmaf(k.du, Lu, ku * Ru);
                                  f0v[i][cc] = fmaf(k.dv, Lv, kv * Rv);
                              });
        hk ^= 1;
    };
    eval0();
    float rmax = 0.f;
    if (adaptive) {
#pragma unroll
        for (int i = 0; i < TY; ++i)
#pragma unroll
            for (int cc = 0; cc < TX; ++cc)
                rmax = fmaxf(rmax, gersh_cell<MODEL>(y0u[i][cc] + k.u0, y0v[i][cc] + k.v0, ncount(i, cc), k));
    }
    {
        float dummy = 0.f;
        block_reduce2(dummy, rmax, reinterpret_cast<float *>(red));
    }
    if (tid == 0) {
        c.t = 0.0;
        c.t_end = t_end;
        c.h = run.h0;
        c.h_prev = 0.0;
        c.err_prev = 0.f;
        c.attempts = 0;
        c.n_acc = 0;
        c.n_rej = 0;
        c.n_rhs = 1;
        c.rho = rmax;
        c.s = 0;
        c.s_used = 0;
        c.have_prev = 0;
        c.after_reject = 0;
        c.accept = 0;
        c.done = 0;
        c.fail = 0;
        rkc_plan(c, run, betaS);
    }
    __syncthreads();

    while (!c.done) {
        const int s = c.s;
        const float h = c.hf;
        const float4 *row = tab + (size_t)s * RKC_STRIDE;
        // coefficient row of this s into shared memory (first read after the
        // exchange barrier of stage 2)
        for (int i = tid; i <= s; i += blockDim.x) crow[i] = row[i];
        // stage 1
        {
            const float m1 = row[1].z * h;
#pragma unroll
            for (int i = 0; i < TY; ++i)
#pragma unroll
                for (int cc = 0; cc < TX; ++cc) {
                    d1u[i][cc] = m1 * f0u[i][cc];
                    d1v[i][cc] = m1 * f0v[i][cc];
                    d2u[i][cc] = 0.f;
                    d2v[i][cc] = 0.f;
                }
        }
        // stages 2..s, two per iteration so that the roles of the latest and
        // previous increments alternate without register moves
        for (int j = 2; j <= s; j += 2) {
            rkc_stage<MODEL, G, TY, TX>(ring + hk * (T::HALO_FLOATS / 2), tx, ty, y0u, y0v, f0u, f0v, d1u, d1v, d2u,
                                        d2v, crow, j, h, k);
            hk ^= 1;
            if (j + 1 > s) {
#pragma unroll
                for (int i = 0; i < TY; ++i)
#pragma unroll
                    for (int cc = 0; cc < TX; ++cc) {
                        d1u[i][cc] = d2u[i][cc];
                        d1v[i][cc] = d2v[i][cc];
                    }
                break;
            }
            rkc_stage<MODEL, G, TY, TX>(ring + hk * (T::HALO_FLOATS / 2), tx, ty, y0u, y0v, f0u, f0v, d2u, d2v, d1u,
                                        d1v, crow, j + 1, h, k);
            hk ^= 1;
        }
        // dF(D_s) = F(Y_s) - F_0, error estimate and rho(Y_s)
        float acc = 0.f;
        rmax = 0.f;
        if (adaptive) {
            const float rtol = (float)run.rtol, atol = (float)run.atol, h04 = 0.4f * h;
            tile_exchange<G, TY, TX>(ring + hk * (T::HALO_FLOATS / 2), tx, ty, d1u, d1v);
            tile_apply<G, TY, TX>(
                ring + hk * (T::HALO_FLOATS / 2), tx, ty, d1u, d1v, [&](int i, int cc, float4 nu, float4 nv) {
                    float dRu = 0.f, dRv = 0.f;
                    if (MODEL != RD_DIFF)
                        rhs_dparts<MODEL>(y0u[i][cc], y0v[i][cc], d1u[i][cc], d1v[i][cc], k, dRu, dRv);
                    const float dFu = fmaf(k.du, lap5(d1u[i][cc], nu), ku * dRu);
                    const float dFv = fmaf(k.dv, lap5(d1v[i][cc], nv), kv * dRv);
                    // est = (12 (Y_0 - Y_s) + 6 h (F_0 + F_s)) / 15
                    //     = -0.8 D_s + 0.4 h (2 F_0 + dF(D_s))
                    const float eu = fmaf(-0.8f, d1u[i][cc], h04 * fmaf(2.f, f0u[i][cc], dFu));
                    const float ev = fmaf(-0.8f, d1v[i][cc], h04 * fmaf(2.f, f0v[i][cc], dFv));
                    const float U0 = y0u[i][cc] + k.u0, V0 = y0v[i][cc] + k.v0;
                    const float Us = (y0u[i][cc] + d1u[i][cc]) + k.u0, Vs = (y0v[i][cc] + d1v[i][cc]) + k.v0;
                    const float qu = __fdividef(eu, fmaf(rtol, fmaxf(fabsf(U0), fabsf(Us)), atol));
                    const float qv = __fdividef(ev, fmaf(rtol, fmaxf(fabsf(V0), fabsf(Vs)), atol));
                    acc = fmaf(qu, qu, fmaf(qv, qv, acc));
                    rmax = fmaxf(rmax, gersh_cell<MODEL>(Us, Vs, ncount(i, cc), k));
                });
            hk ^= 1;
        }
        float ss = acc;
        block_reduce2(ss, rmax, reinterpret_cast<float *>(red));
        if (tid == 0) {
            c.rho_new = rmax;
            rkc_decide(c, run, betaS, ss, M);
        }
        __syncthreads();
        if (c.accept) {
            // (y0 + c0) + D_s, compensated: TwoSum of y0 and D_s, its error
            // added to c0, renormalised
#pragma unroll
            for (int i = 0; i < TY; ++i)
#pragma unroll
                for (int cc = 0; cc < TX; ++cc) {
                    const int node = (ty * TY + i) * G + tx * TX + cc;
                    {
                        const float sw = y0u[i][cc] + d1u[i][cc], bp = sw - y0u[i][cc];
                        const float e = (y0u[i][cc] - (sw - bp)) + (d1u[i][cc] - bp);
                        const float lo = c0[node] + e;
                        y0u[i][cc] = sw + lo;
                        c0[node] = lo - (y0u[i][cc] - sw);
                    }
                    {
                        const float sw = y0v[i][cc] + d1v[i][cc], bp = sw - y0v[i][cc];
                        const float e = (y0v[i][cc] - (sw - bp)) + (d1v[i][cc] - bp);
                        const float lo = c0[G * G + node] + e;
                        y0v[i][cc] = sw + lo;
                        c0[G * G + node] = lo - (y0v[i][cc] - sw);
                    }
                }
            // F_0 of the new state afresh (not F_0 + dF(D_s)), so the run
            // keeps solving the discrete system of the state it holds
            if (!c.done) eval0();
        }
    }
    {
        CoefF cf{};
        cf.u0 = k.u0;
        cf.v0 = k.v0;
        tile_from_state<MODEL, TY, TX>(y0u, y0v, cf);
    }
    tile_store<G, TY, TX>(base, tx, ty, y0u, y0v);
    if (tid == 0) {
        if (stats) {
            int64_t *st = stats + 4 * (int64_t)r;
            st[0] = c.n_acc;
            st[1] = c.n_rej;
            st[2] = c.n_rhs;
            st[3] = c.s_used;
        }
        if (c.fail == 1) atomicOr(status, (unsigned)ST_STEPFAIL);
        if (c.fail == 2) atomicOr(status, (unsigned)ST_NONFINITE);
    }
    residual_from_global<MODEL, G>(base, p0, p1, p2, p3, residual, status, r, ring);
}

// Tile shapes (TY x TX nodes per thread), per grid side; every shape runs
// the same per-node arithmetic, so all give bit-identical fields.
//   G = 32: 0 = 2 x 1 (512 threads), 1 = 4 x 1 (256), 2 = 2 x 2 (256)
//   G = 64: 0 = 4 x 2 (512 threads), 1 = 4 x 4 (256, default), 2 = 2 x 4 (512)
constexpr int RKC_NVAR = 3;
template <int G, int V> struct RkcShape;
template <> struct RkcShape<32, 0> { static constexpr int TY = 2, TX = 1; };
template <> struct RkcShape<32, 1> { static constexpr int TY = 4, TX = 1; };
template <> struct RkcShape<32, 2> { static constexpr int TY = 2, TX = 2; };
template <> struct RkcShape<64, 0> { static constexpr int TY = 4, TX = 2; };
template <> struct RkcShape<64, 1> { static constexpr int TY = 4, TX = 4; };
template <> struct RkcShape<64, 2> { static constexpr int TY = 2, TX = 4; };
// defaults: FHN 64x64 x 128, fixed 16-stage schedule on B300: 4 x 4 took
// 0.668 us per stage, 4 x 2 0.705, 2 x 4 0.736
static int g_rkc_var[2] = {0, 1};   // [G == 64]

int rkc_n_variants() { return RKC_NVAR; }
bool rkc_set_variant(int G, int v) {
    if ((G != 32 && G != 64) || v < 0 || v >= RKC_NVAR) return false;
    g_rkc_var[G == 64] = v;
    return true;
}
int rkc_get_variant(int G) { return (G == 32 || G == 64) ? g_rkc_var[G == 64] : -1; }

template <int MODEL, int G, int V>
static rd_status launch_rkc_mg(const GroupDev &g, const float4 *tab, const double *beta, float *fields,
                               const RkcRun &run, int64_t *stats, double *residual, uint32_t *status,
                               cudaStream_t s) {
    constexpr int TY = RkcShape<G, V>::TY, TX = RkcShape<G, V>::TX;
    using T = Tiling<G, TY, TX>;
    const size_t smem = rkc_smem<G, TY, TX>();
    auto kern = rd_rkc_kernel<MODEL, G, TY, TX>;
    RD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const double t_end = run.t_end > 0.0 ? run.t_end : g.dt * (double)g.n_steps;
    kern<<<g.n_real, T::NT, smem, s>>>(fields, g.field_offset, make_rkc_k(g), run, t_end, tab, beta,
                                       stats ? stats + 4 * g.real_base : nullptr, g.p[0], g.p[1], g.p[2], g.p[3],
                                       residual ? residual + 2 * g.real_base : nullptr, status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL>
static rd_status launch_rkc_m(const GroupDev &g, const float4 *tab, const double *beta, float *fields,
                              const RkcRun &run, int64_t *stats, double *residual, uint32_t *status,
                              cudaStream_t s) {
    const int v = rkc_get_variant(g.G);
    if (g.G == 32) {
        if (v == 1) return launch_rkc_mg<MODEL, 32, 1>(g, tab, beta, fields, run, stats, residual, status, s);
        if (v == 2) return launch_rkc_mg<MODEL, 32, 2>(g, tab, beta, fields, run, stats, residual, status, s);
        return launch_rkc_mg<MODEL, 32, 0>(g, tab, beta, fields, run, stats, residual, status, s);
    }
    if (g.G == 64) {
        if (v == 1) return launch_rkc_mg<MODEL, 64, 1>(g, tab, beta, fields, run, stats, residual, status, s);
        if (v == 2) return launch_rkc_mg<MODEL, 64, 2>(g, tab, beta, fields, run, stats, residual, status, s);
        return launch_rkc_mg<MODEL, 64, 0>(g, tab, beta, fields, run, stats, residual, status, s);
    }
    return RD_ERR_UNSUPPORTED;
}

bool rkc_supported(const GroupDev &g) {
    if (g.model == RD_RDODE) return rkc1d_supported(g);
    return g.G == 32 || g.G == 64 || g.G == 128;
}

rd_status launch_rkc_group(const GroupDev &g, const float4 *tab, const double *beta, float *fields,
                           const rd_rkc_opts &o, int64_t *stats, double *residual, uint32_t *status,
                           cudaStream_t s) {
    if (!tab || !beta) return RD_ERR_UNSUPPORTED;
    if (g.model == RD_RDODE) return launch_rkc1d_group(g, tab, beta, fields, o, stats, residual, status, s);
    RkcRun run{o.t_end, o.h0, o.rtol, o.atol, o.s_max, o.s_fixed, o.n_fixed, o.max_attempts};
    if (g.G == 128) return launch_rkc_cluster_group(g, fields, run, tab, beta, stats, residual, status, s);
    switch (g.model) {
        case RD_FHN: return launch_rkc_m<RD_FHN>(g, tab, beta, fields, run, stats, residual, status, s);
        case RD_GM: return launch_rkc_m<RD_GM>(g, tab, beta, fields, run, stats, residual, status, s);
        case RD_DIFF: return launch_rkc_m<RD_DIFF>(g, tab, beta, fields, run, stats, residual, status, s);
        case RD_BZ: return launch_rkc_m<RD_BZ>(g, tab, beta, fields, run, stats, residual, status, s);
        default: return RD_ERR_INVALID_ARG;
    }
}

}  // namespace rdcil
