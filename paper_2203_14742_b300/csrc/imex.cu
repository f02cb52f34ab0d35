// Semi-implicit (IMEX) Euler integration of the batched 2-D reaction-
// diffusion systems: diffusion implicit, reaction explicit,
//   (I - dt D_s L_h) w_s^{n+1} = w_s^n + dt R_s(u^n, v^n),   s = u, v,
// with L_h the 5-point Laplacian with mirrored Neumann ghosts (App. B.1.1;
// Sec. 4.1 kinetics).  Sec. 5.1 and App. B.2 weigh explicit stepping
// against implicit stepping with linear solves; this is the implicit
// treatment of the stiff (diffusive) part alone, so the time step is bound
// by the reaction rather than by h^2 / (4 D).
//
// The solve.  With ghost = edge node the 1-D second difference is
// diagonalised by the orthonormal DCT-II,
//   C[p][x] = a_p cos(pi p (2x + 1) / (2G)),  a_0 = sqrt(1/G), a_p = sqrt(2/G),
// with eigenvalue -mu_p, mu_p = 4 sin^2(pi p / (2G)) (times (G-1)^2), so
//   w^{n+1} = C^T ((C b C^T) o S) C,   S[q][p] = 1 / (1 + dt D (G-1)^2 (mu_p + mu_q)),
// b the explicit right side: four dense G x G x G products per species and
// step, exact up to rounding (no iteration).
//
// Increment form.  Subtracting (I - dt D L_h) w^n from both sides gives the
// same step as
//   (I - dt D_s L_h) d_s = dt F_s(w^n),   w_s^{n+1} = w_s^n + d_s,
// F = D L_h w + R the explicit right-hand side, so the transforms carry the
// small increment and their FP32 rounding is relative to it rather than to
// the field (with b itself the rounding of four products of the whole field
// per step built up to 2e-5 over 300 FHN steps); at a steady state F = 0
// and the state stays in place.
//
// B300 design.  One CTA per realisation keeps both species, the transform
// matrices C and C^T, both divisor tables and, per species, an increment
// and a product buffer in shared memory for the whole run (G = 64: 174 KB); nothing goes to HBM between
// steps.  The two halves of the block take the two species' products side
// by side; a thread accumulates a 4 x 4 output tile in FP32 FMAs from one
// broadcast float4 of the left operand (stored k-major) and one float4 of
// the right operand per k.  The first and third product store their
// result transposed, which is the k-major operand the next product wants;
// the divisors are applied in the second product's epilogue and the
// increment is added to the state in the fourth's.  The tables
// are computed once per G in FP64 (cospi, sinpi) and rounded once; the
// divisors are formed per CTA in FP32 from mu.  GM and BZ states are the
// deviation from the FP32 equilibrium (the constant lies in mode (0, 0),
// whose divisor is 1, so the solve commutes with the shift), which keeps
// the transforms' rounding relative to the pattern rather than to the
// equilibrium value.
#include <cmath>
#include <mutex>
#include <cooperative_groups.h>
#include "common.cuh"
#include "tile.cuh"

namespace rdcil {

// tab = [C (G x G) | C^T (G x G) | mu (G)], row-major, FP32.
__global__ void imex_table_kernel(int G, float *__restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G * G) {
        const int p = i / G, x = i - p * G;
        const double a = p == 0 ? sqrt(1.0 / (double)G) : sqrt(2.0 / (double)G);
        // p (2x + 1) / (2G) is exact in FP64 for the grid sides used
        const float c = (float)(a * cospi((double)(p * (2 * x + 1)) / (double)(2 * G)));
        tab[p * G + x] = c;
        tab[G * G + x * G + p] = c;
    }
    if (i < G) {
        const double s = sinpi((double)i / (double)(2 * G));
        tab[2 * G * G + i] = (float)(4.0 * s * s);
    }
}

// dt F(w) at one node from the neighbour sums su = (N + S) + (W + E) of the
// state registers (deviation form for GM and BZ, as in euler_cell; the
// Laplacian of a deviation is that of the field):
//   FHN: d_u = cu (su - 4u) + dt (u - u^3 - v),   d_v = cv (sv - 4v) + dt eps (u - a v)
//   GM:  d_a = cu (sa - 4a) + k2 U (a - mu b + e0) / V,
//        d_b = cv (sb - 4b) + k2 (a (a + 2 u0) - b + e1)
//   BZ:  d_a = cu (sa - 4a) + dt (e0 + c1 a + P),  d_b = cv (sb - 4b) + dt (-e0 + c2 a - P)
// with cu = Du dt (G-1)^2, cv = Dv dt (G-1)^2.
template <int MODEL>
__device__ __forceinline__ void incr(float u, float v, float su, float sv, const CoefF &c, float &du, float &dv) {
    const float lu = c.cu * fmaf(-4.f, u, su), lv = c.cv * fmaf(-4.f, v, sv);
    if (MODEL == RD_FHN) {
        const float ru = fmaf(-u * u, u, u - v);
        const float rv = fmaf(-c.k3, v, u);
        du = fmaf(c.k1, ru, lu);
        dv = fmaf(c.k2, rv, lv);
    } else if (MODEL == RD_GM) {
        const float a = u, b = v;
        const float U = a + c.u0, V = b + c.v0;
        const float t = fmaf(-c.k3, b, a + c.e0);
        const float f = __fdividef(U * t, V);
        du = fmaf(c.k2, f, lu);
        dv = fmaf(c.k2, fmaf(a, a + c.tu0, c.e1 - b), lv);
    } else if (MODEL == RD_BZ) {
        const float a = u, b = v;
        const float U = a + c.u0;
        const float P = fmaf(c.v0 * a, a, (U * U) * b);
        const float f = fmaf(c.c1, a, c.e0 + P);
        const float g = fmaf(c.c2, a, -c.e0 - P);
        du = fmaf(c.k1, f, lu);
        dv = fmaf(c.k1, g, lv);
    } else {
        du = lu;
        dv = lv;
    }
}

// dt F of the four nodes (y, x..x+3) of both species into Xu, Xv, with
// mirrored ghosts at the edges.
template <int MODEL, int G>
__device__ __forceinline__ void incr4(const float *__restrict__ Wu, const float *__restrict__ Wv,
                                      float *__restrict__ Xu, float *__restrict__ Xv, int y, int x,
                                      const CoefF &cf) {
    constexpr int LD = G + 4;
    const int o = y * LD + x, on = (y > 0 ? o - LD : o), os = (y < G - 1 ? o + LD : o);
    float su[4], sv[4], cu[4], cv[4];
    {
        const float4 c = *reinterpret_cast<const float4 *>(Wu + o);
        const float4 n = *reinterpret_cast<const float4 *>(Wu + on);
        const float4 s = *reinterpret_cast<const float4 *>(Wu + os);
        const float w = x > 0 ? Wu[o - 1] : c.x, e = x + 4 < G ? Wu[o + 4] : c.w;
        cu[0] = c.x; cu[1] = c.y; cu[2] = c.z; cu[3] = c.w;
        su[0] = (n.x + s.x) + (w + c.y);
        su[1] = (n.y + s.y) + (c.x + c.z);
        su[2] = (n.z + s.z) + (c.y + c.w);
        su[3] = (n.w + s.w) + (c.z + e);
    }
    {
        const float4 c = *reinterpret_cast<const float4 *>(Wv + o);
        const float4 n = *reinterpret_cast<const float4 *>(Wv + on);
        const float4 s = *reinterpret_cast<const float4 *>(Wv + os);
        const float w = x > 0 ? Wv[o - 1] : c.x, e = x + 4 < G ? Wv[o + 4] : c.w;
        cv[0] = c.x; cv[1] = c.y; cv[2] = c.z; cv[3] = c.w;
        sv[0] = (n.x + s.x) + (w + c.y);
        sv[1] = (n.y + s.y) + (c.x + c.z);
        sv[2] = (n.z + s.z) + (c.y + c.w);
        sv[3] = (n.w + s.w) + (c.z + e);
    }
    float du[4], dv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) incr<MODEL>(cu[j], cv[j], su[j], sv[j], cf, du[j], dv[j]);
    *reinterpret_cast<float4 *>(Xu + o) = make_float4(du[0], du[1], du[2], du[3]);
    *reinterpret_cast<float4 *>(Xv + o) = make_float4(dv[0], dv[1], dv[2], dv[3]);
}

// out[r][c] = sum_k At[k][r] B[k][c] over a G x G product in shared memory
// (leading dimension G + 4).  The calling thread owns a TM x TN tile: rows
// 4ty + (i mod 4) + (i div 4) G/2 and columns 4tx + (j mod 4) + (j div 4) G/2,
// so each of its 128-bit loads, with its warp's neighbours, covers
// consecutive banks.  Per k: TM/4 broadcast float4 of the left operand
// (k-major) and TN/4 float4 of the right one for TM TN FMAs.  TRANS stores
// out[c][r] instead; SCALE multiplies by Sc[r][c] on the way out; ADD adds
// the result to out.
template <int G, int TM, int TN, bool TRANS, bool SCALE, bool ADD = false>
__device__ __forceinline__ void imex_mm(const float *__restrict__ At, const float *__restrict__ B,
                                        float *__restrict__ out, const float *__restrict__ Sc, int ty, int tx) {
    constexpr int LD = G + 4, H = G / 2;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    const float *pa = At + 4 * ty, *pb = B + 4 * tx;
#pragma unroll 4
    for (int k = 0; k < G; ++k) {
        float av[TM], bv[TN];
#pragma unroll
        for (int h = 0; h < TM / 4; ++h) {
            const float4 a = *reinterpret_cast<const float4 *>(pa + k * LD + h * H);
            av[4 * h] = a.x; av[4 * h + 1] = a.y; av[4 * h + 2] = a.z; av[4 * h + 3] = a.w;
        }
#pragma unroll
        for (int h = 0; h < TN / 4; ++h) {
            const float4 b = *reinterpret_cast<const float4 *>(pb + k * LD + h * H);
            bv[4 * h] = b.x; bv[4 * h + 1] = b.y; bv[4 * h + 2] = b.z; bv[4 * h + 3] = b.w;
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (TRANS) {
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = 4 * tx + (j & 3) + (j >> 2) * H;
#pragma unroll
            for (int h = 0; h < TM / 4; ++h)
                *reinterpret_cast<float4 *>(out + c * LD + 4 * ty + h * H) =
                    make_float4(acc[4 * h][j], acc[4 * h + 1][j], acc[4 * h + 2][j], acc[4 * h + 3][j]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int r = 4 * ty + (i & 3) + (i >> 2) * H;
#pragma unroll
            for (int h = 0; h < TN / 4; ++h) {
                const int o = r * LD + 4 * tx + h * H;
                float4 v = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
                if (SCALE) {
                    const float4 sc = *reinterpret_cast<const float4 *>(Sc + o);
                    v.x *= sc.x; v.y *= sc.y; v.z *= sc.z; v.w *= sc.w;
                }
                if (ADD) {
                    const float4 w = *reinterpret_cast<const float4 *>(out + o);
                    v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
                }
                *reinterpret_cast<float4 *>(out + o) = v;
            }
        }
    }
}

template <int G>
constexpr size_t imex_smem() { return sizeof(float) * 10 * (size_t)G * (G + 4); }

template <int MODEL, int G, int TM, int TN>
__global__ void __launch_bounds__(2 * (G / TM) * (G / TN))
rd_imex_kernel(float *__restrict__ fields, int64_t field_offset, CoefF cf, float a_u, float a_v,
               const float *__restrict__ tab, int64_t steps, double p0, double p1, double p2, double p3,
               double *__restrict__ residual, uint32_t *__restrict__ status) {
    constexpr int LD = G + 4, Q = G / 4, QX = G / TN, NS = (G / TM) * QX, NT = 2 * NS, BUF = G * LD;
    extern __shared__ __align__(16) float sm[];
    float *sC = sm, *sCT = sC + BUF, *sS = sCT + BUF, *sW = sS + 2 * BUF, *sX = sW + 2 * BUF, *sT = sX + 2 * BUF;
    const int tid = threadIdx.x, r = blockIdx.x;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;
    const float *mu = tab + 2 * G * G;
    for (int q = tid; q < G * Q; q += NT) {
        const int y = q / Q, x = (q - y * Q) * 4;
        *reinterpret_cast<float4 *>(sC + y * LD + x) = *reinterpret_cast<const float4 *>(tab + y * G + x);
        *reinterpret_cast<float4 *>(sCT + y * LD + x) = *reinterpret_cast<const float4 *>(tab + G * G + y * G + x);
        float4 u = *reinterpret_cast<const float4 *>(base + y * G + x);
        float4 v = *reinterpret_cast<const float4 *>(base + G * G + y * G + x);
        to_state<MODEL>(u.x, v.x, cf);
        to_state<MODEL>(u.y, v.y, cf);
        to_state<MODEL>(u.z, v.z, cf);
        to_state<MODEL>(u.w, v.w, cf);
        *reinterpret_cast<float4 *>(sW + y * LD + x) = u;
        *reinterpret_cast<float4 *>(sW + BUF + y * LD + x) = v;
        float su[4], sv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float m = mu[y] + mu[x + j];
            su[j] = 1.f / fmaf(a_u, m, 1.f);
            sv[j] = 1.f / fmaf(a_v, m, 1.f);
        }
        *reinterpret_cast<float4 *>(sS + y * LD + x) = make_float4(su[0], su[1], su[2], su[3]);
        *reinterpret_cast<float4 *>(sS + BUF + y * LD + x) = make_float4(sv[0], sv[1], sv[2], sv[3]);
    }
    __syncthreads();
    const int sp = tid / NS, l = tid - sp * NS, ty = l / QX, tx = l - ty * QX;
    float *F = sW + sp * BUF, *X = sX + sp * BUF, *T = sT + sp * BUF;
    const float *S = sS + sp * BUF;
    for (int64_t n = 0; n < steps; ++n) {
        for (int q = tid; q < G * Q; q += NT) {
            const int y = q / Q, x = (q - y * Q) * 4;
            incr4<MODEL, G>(sW, sW + BUF, sX, sX + BUF, y, x, cf);   // dt F(w^n)
        }
        __syncthreads();
        imex_mm<G, TM, TN, true, false>(sCT, X, T, nullptr, ty, tx);        // (C dtF)^T
        __syncthreads();
        imex_mm<G, TM, TN, false, true>(T, sCT, X, S, ty, tx);              // (C dtF C^T) o S
        __syncthreads();
        imex_mm<G, TM, TN, true, false>(sC, X, T, nullptr, ty, tx);         // (C^T .)^T
        __syncthreads();
        imex_mm<G, TM, TN, false, false, true>(T, sC, F, nullptr, ty, tx);  // w += C^T . C
        __syncthreads();
    }
    for (int q = tid; q < G * Q; q += NT) {
        const int y = q / Q, x = (q - y * Q) * 4;
        float4 u = *reinterpret_cast<const float4 *>(sW + y * LD + x);
        float4 v = *reinterpret_cast<const float4 *>(sW + BUF + y * LD + x);
        from_state<MODEL>(u.x, v.x, cf);
        from_state<MODEL>(u.y, v.y, cf);
        from_state<MODEL>(u.z, v.z, cf);
        from_state<MODEL>(u.w, v.w, cf);
        *reinterpret_cast<float4 *>(base + y * G + x) = u;
        *reinterpret_cast<float4 *>(base + G * G + y * G + x) = v;
    }
    residual_from_global<MODEL, G>(base, p0, p1, p2, p3, residual, status, r, sC);
}

// floats of the full-product table (C, C^T, divisor eigenvalues) at G
// (G = 32, 64; the G = 128 cluster kernel uses the even/odd table alone)
size_t imex_table_floats(int G) { return G == 128 ? 0 : 2 * (size_t)G * G + G; }

// ---------------------------------------------------------------------------
// Even/odd split.  C[p][G-1-x] = (-1)^p C[p][x], so with the spectrum held in
// the order m = (even p ascending, odd p ascending), C'[m] = C[p(m)], every
// product is two half-length sums:
//   forward (C' Y)[m] = sum_{k<G/2} C'[m][k] (Y[k] +- Y[G-1-k])   (+ for m < G/2)
//   inverse (C'^T Z)[y], [G-1-y] = A_e +- A_o,  A_e = sum_{k<G/2} C'[k][y] Z[k],
//                                               A_o = sum_{k<G/2} C'[k+G/2][y] Z[k+G/2]
// (y < G/2), half the FMAs of the full products; the divisors are applied
// in the permuted order.  Tables: Ch[k][m] = C'[m][k] (k < G/2, ld G + 4)
// and Cl[m][y] = C'[m][y] (y < G/2, ld G/2 + 4).  Every product gives each
// thread 32 outputs from 16 accumulator pairs of float4 loads per k.
// ---------------------------------------------------------------------------
__global__ void imex_eo_table_kernel(int G, float *__restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int H = G / 2;
    if (i < G * H) {
        const int m = i / H, y = i - m * H;
        const int p = m < H ? 2 * m : 2 * (m - H) + 1;
        const double a = p == 0 ? sqrt(1.0 / (double)G) : sqrt(2.0 / (double)G);
        const float c = (float)(a * cospi((double)(p * (2 * y + 1)) / (double)(2 * G)));
        tab[y * G + m] = c;           // Ch: [k = y < H][m]
        tab[H * G + m * H + y] = c;   // Cl: [m][y < H]
    }
    if (i < G) {
        const int p = i < H ? 2 * i : 2 * (i - H) + 1;
        const double s = sinpi((double)p / (double)(2 * G));
        tab[2 * H * G + i] = (float)(4.0 * s * s);   // mu in the permuted order
    }
}

__device__ __forceinline__ void f4a(float (&d)[4], float4 v) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }

// The transposed buffer T holds float4 slot s of row c at slot
// s ^ ((c / 4) mod 8): the forward and inverse row products write rows
// 4tx + j of a warp's lanes, which with ld = G + 4 would fall on two bank
// quads; the swizzle spreads eight lanes over eight.  Readers apply the same
// map.
__device__ __forceinline__ int swz(int c, int s) { return s ^ ((c >> 2) & 7); }

// forward along the rows' index: T[c][m] = sum_k Ch[k][m] (Y[k][c] +- Y[G-1-k][c])
// (stored transposed); thread: m = 4ty + i (+ G/2), c = 4tx + j
template <int G>
__device__ __forceinline__ void eo_fwd_rows(const float *__restrict__ Ch, const float *__restrict__ Y,
                                           float *__restrict__ T, int l) {
    constexpr int LD = G + 4, H = G / 2;
    const int tx = l % (G / 4), ty = l / (G / 4);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        float ae[4], ao[4], y1[4], y2[4];
        f4a(ae, *reinterpret_cast<const float4 *>(Ch + k * LD + 4 * ty));
        f4a(ao, *reinterpret_cast<const float4 *>(Ch + k * LD + 4 * ty + H));
        f4a(y1, *reinterpret_cast<const float4 *>(Y + k * LD + 4 * tx));
        f4a(y2, *reinterpret_cast<const float4 *>(Y + (G - 1 - k) * LD + 4 * tx));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float e = y1[j] + y2[j], o = y1[j] - y2[j];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][j] = fmaf(ae[i], e, acc[i][j]);
                acc[4 + i][j] = fmaf(ao[i], o, acc[4 + i][j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = 4 * tx + j;
        float *row = T + c * LD;
        *reinterpret_cast<float4 *>(row + 4 * swz(c, ty)) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        *reinterpret_cast<float4 *>(row + 4 * swz(c, ty + H / 4)) =
            make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
    }
}

// forward along the columns' index, divisors applied:
// Z[r][m] = S[r][m] sum_k (T[k][r] +- T[G-1-k][r]) Ch[k][m]; thread: r = 4ty + i, m = 4tx + j (+ G/2)
template <int G>
__device__ __forceinline__ void eo_fwd_cols(const float *__restrict__ T, const float *__restrict__ Ch,
                                           float *__restrict__ Z, const float *__restrict__ S, int l) {
    constexpr int LD = G + 4, H = G / 2;
    const int tx = l % (G / 8), ty = l / (G / 8);
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        float t1[4], t2[4], be[4], bo[4];
        f4a(t1, *reinterpret_cast<const float4 *>(T + k * LD + 4 * swz(k, ty)));
        f4a(t2, *reinterpret_cast<const float4 *>(T + (G - 1 - k) * LD + 4 * swz(G - 1 - k, ty)));
        f4a(be, *reinterpret_cast<const float4 *>(Ch + k * LD + 4 * tx));
        f4a(bo, *reinterpret_cast<const float4 *>(Ch + k * LD + 4 * tx + H));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float e = t1[i] + t2[i], o = t1[i] - t2[i];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[i][j] = fmaf(e, be[j], acc[i][j]);
                acc[i][4 + j] = fmaf(o, bo[j], acc[i][4 + j]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int o0 = (4 * ty + i) * LD + 4 * tx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 sc = *reinterpret_cast<const float4 *>(S + o0 + h * H);
            *reinterpret_cast<float4 *>(Z + o0 + h * H) =
                make_float4(acc[i][4 * h] * sc.x, acc[i][4 * h + 1] * sc.y, acc[i][4 * h + 2] * sc.z,
                            acc[i][4 * h + 3] * sc.w);
        }
    }
}

// inverse along the rows' index: T[c][y], T[c][G-1-y] = A_e +- A_o with
// A_e = sum_k Cl[k][y] Z[k][c], A_o = sum_k Cl[k+G/2][y] Z[k+G/2][c]
// (stored transposed); thread: y = 4ty + i (< G/2), c = 4tx + j
template <int G>
__device__ __forceinline__ void eo_inv_rows(const float *__restrict__ Cl, const float *__restrict__ Z,
                                           float *__restrict__ T, int l) {
    constexpr int LD = G + 4, H = G / 2, LDH = H + 4;
    const int tx = l % (G / 4), ty = l / (G / 4);
    float E[4][4], O[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) E[i][j] = O[i][j] = 0.f;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        float ae[4], ao[4], z1[4], z2[4];
        f4a(ae, *reinterpret_cast<const float4 *>(Cl + k * LDH + 4 * ty));
        f4a(ao, *reinterpret_cast<const float4 *>(Cl + (k + H) * LDH + 4 * ty));
        f4a(z1, *reinterpret_cast<const float4 *>(Z + k * LD + 4 * tx));
        f4a(z2, *reinterpret_cast<const float4 *>(Z + (k + H) * LD + 4 * tx));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                E[i][j] = fmaf(ae[i], z1[j], E[i][j]);
                O[i][j] = fmaf(ao[i], z2[j], O[i][j]);
            }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = 4 * tx + j;
        float *row = T + c * LD;
        *reinterpret_cast<float4 *>(row + 4 * swz(c, ty)) =
            make_float4(E[0][j] + O[0][j], E[1][j] + O[1][j], E[2][j] + O[2][j], E[3][j] + O[3][j]);
        *reinterpret_cast<float4 *>(row + 4 * swz(c, G / 4 - 1 - ty)) =
            make_float4(E[3][j] - O[3][j], E[2][j] - O[2][j], E[1][j] - O[1][j], E[0][j] - O[0][j]);
    }
}

// inverse along the columns' index, added to the state: W[r][x], W[r][G-1-x]
// += B_e +- B_o, B_e = sum_k T[k][r] Cl[k][x], B_o = sum_k T[k+G/2][r] Cl[k+G/2][x];
// thread: r = 4ty + i, x = 4tx + j (< G/2)
template <int G>
__device__ __forceinline__ void eo_inv_cols(const float *__restrict__ T, const float *__restrict__ Cl,
                                           float *__restrict__ W, int l) {
    constexpr int LD = G + 4, H = G / 2, LDH = H + 4;
    const int tx = l % (H / 4), ty = l / (H / 4);
    float E[4][4], O[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) E[i][j] = O[i][j] = 0.f;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        float t1[4], t2[4], b1[4], b2[4];
        f4a(t1, *reinterpret_cast<const float4 *>(T + k * LD + 4 * swz(k, ty)));
        f4a(t2, *reinterpret_cast<const float4 *>(T + (k + H) * LD + 4 * swz(k + H, ty)));
        f4a(b1, *reinterpret_cast<const float4 *>(Cl + k * LDH + 4 * tx));
        f4a(b2, *reinterpret_cast<const float4 *>(Cl + (k + H) * LDH + 4 * tx));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                E[i][j] = fmaf(t1[i], b1[j], E[i][j]);
                O[i][j] = fmaf(t2[i], b2[j], O[i][j]);
            }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float *row = W + (4 * ty + i) * LD;
        float4 a = *reinterpret_cast<const float4 *>(row + 4 * tx);
        a.x += E[i][0] + O[i][0]; a.y += E[i][1] + O[i][1]; a.z += E[i][2] + O[i][2]; a.w += E[i][3] + O[i][3];
        *reinterpret_cast<float4 *>(row + 4 * tx) = a;
        float4 b = *reinterpret_cast<const float4 *>(row + G - 4 - 4 * tx);
        b.x += E[i][3] - O[i][3]; b.y += E[i][2] - O[i][2]; b.z += E[i][1] - O[i][1]; b.w += E[i][0] - O[i][0];
        *reinterpret_cast<float4 *>(row + G - 4 - 4 * tx) = b;
    }
}

template <int G>
constexpr size_t imex_eo_smem() {
    return sizeof(float) * ((size_t)(G / 2) * (G + 4) + (size_t)G * (G / 2 + 4) + 8 * (size_t)G * (G + 4));
}

template <int MODEL, int G>
__global__ void __launch_bounds__(G * G / 16)
rd_imex_eo_kernel(float *__restrict__ fields, int64_t field_offset, CoefF cf, float a_u, float a_v,
                  const float *__restrict__ tab, int64_t steps, double p0, double p1, double p2, double p3,
                  double *__restrict__ residual, uint32_t *__restrict__ status) {
    constexpr int LD = G + 4, H = G / 2, LDH = H + 4, Q = G / 4, NS = G * G / 32, NT = 2 * NS, BUF = G * LD;
    extern __shared__ __align__(16) float sm[];
    float *sCh = sm, *sCl = sCh + H * LD, *sS = sCl + G * LDH, *sW = sS + 2 * BUF, *sX = sW + 2 * BUF,
          *sT = sX + 2 * BUF;
    const int tid = threadIdx.x, r = blockIdx.x;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;
    const float *mu = tab + 2 * H * G;
    for (int q = tid; q < H * Q; q += NT) {   // Ch: H rows of G
        const int y = q / Q, x = (q - y * Q) * 4;
        *reinterpret_cast<float4 *>(sCh + y * LD + x) = *reinterpret_cast<const float4 *>(tab + y * G + x);
    }
    for (int q = tid; q < G * (H / 4); q += NT) {   // Cl: G rows of H
        const int y = q / (H / 4), x = (q - y * (H / 4)) * 4;
        *reinterpret_cast<float4 *>(sCl + y * LDH + x) = *reinterpret_cast<const float4 *>(tab + H * G + y * H + x);
    }
    for (int q = tid; q < G * Q; q += NT) {
        const int y = q / Q, x = (q - y * Q) * 4;
        float4 u = *reinterpret_cast<const float4 *>(base + y * G + x);
        float4 v = *reinterpret_cast<const float4 *>(base + G * G + y * G + x);
        to_state<MODEL>(u.x, v.x, cf);
        to_state<MODEL>(u.y, v.y, cf);
        to_state<MODEL>(u.z, v.z, cf);
        to_state<MODEL>(u.w, v.w, cf);
        *reinterpret_cast<float4 *>(sW + y * LD + x) = u;
        *reinterpret_cast<float4 *>(sW + BUF + y * LD + x) = v;
        float su[4], sv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float m = mu[y] + mu[x + j];
            su[j] = 1.f / fmaf(a_u, m, 1.f);
            sv[j] = 1.f / fmaf(a_v, m, 1.f);
        }
        *reinterpret_cast<float4 *>(sS + y * LD + x) = make_float4(su[0], su[1], su[2], su[3]);
        *reinterpret_cast<float4 *>(sS + BUF + y * LD + x) = make_float4(sv[0], sv[1], sv[2], sv[3]);
    }
    __syncthreads();
    const int sp = tid / NS, l = tid - sp * NS;
    float *F = sW + sp * BUF, *X = sX + sp * BUF, *T = sT + sp * BUF;
    const float *S = sS + sp * BUF;
    for (int64_t n = 0; n < steps; ++n) {
        for (int q = tid; q < G * Q; q += NT) {
            const int y = q / Q, x = (q - y * Q) * 4;
            incr4<MODEL, G>(sW, sW + BUF, sX, sX + BUF, y, x, cf);   // dt F(w^n)
        }
        __syncthreads();
        eo_fwd_rows<G>(sCh, X, T, l);
        __syncthreads();
        eo_fwd_cols<G>(T, sCh, X, S, l);
        __syncthreads();
        eo_inv_rows<G>(sCl, X, T, l);
        __syncthreads();
        eo_inv_cols<G>(T, sCl, F, l);
        __syncthreads();
    }
    for (int q = tid; q < G * Q; q += NT) {
        const int y = q / Q, x = (q - y * Q) * 4;
        float4 u = *reinterpret_cast<const float4 *>(sW + y * LD + x);
        float4 v = *reinterpret_cast<const float4 *>(sW + BUF + y * LD + x);
        from_state<MODEL>(u.x, v.x, cf);
        from_state<MODEL>(u.y, v.y, cf);
        from_state<MODEL>(u.z, v.z, cf);
        from_state<MODEL>(u.w, v.w, cf);
        *reinterpret_cast<float4 *>(base + y * G + x) = u;
        *reinterpret_cast<float4 *>(base + G * G + y * G + x) = v;
    }
    residual_from_global<MODEL, G>(base, p0, p1, p2, p3, residual, status, r, sCh);
}

// ---------------------------------------------------------------------------
// G = 128: one 4-CTA cluster per realisation.  The even/odd kernel's shared
// working set at this side (about 600 KB) exceeds one SM, so the grid's rows
// are split: CTA c of the cluster owns rows y in [32c, 32c + 32) of both
// species (state, increment) and, for the transforms along y, the spectral
// columns m in [32c, 32c + 32).  A step:
//   1. dt F of its rows, from the state and two halo rows, stored x-major;
//   2. forward along x (local, full rows): Xh[y][m], sent block by block to
//      the CTA owning column block m / 32 (distributed shared memory), which
//      gathers all 128 rows of its 32 columns;              cluster barrier
//   3. forward along y with the divisors (local): Z[q][m];
//   4. inverse along y (local): Yh[y][m], sent back to the owner of row y,
//      stored m-major;                                        cluster barrier
//   5. inverse along x (local), added to the state; the updated edge rows
//      are written into the neighbours' halo rows;            cluster barrier
// Every product is the even/odd half-length form of the G <= 64 kernel
// (same tables, same permuted spectrum), 32 outputs per thread, the two
// halves of the block on the two species.  Buffer reuse across the barriers:
// a CTA writes another CTA's K (step 2) only after the barrier that follows
// the owner's last read of it (step 3 of the previous step), and the same
// holds for the R buffer (written in 4, read in 5) and the halo rows
// (written in 5, read in 1); the x-major increment of step 1 and R share
// one buffer, since R is written only after the barrier that follows step 2.
// The cluster barriers are hardware barriers that every CTA passes the same
// number of times (no data-dependent control), and a final barrier keeps
// every CTA alive until the others' last remote writes are done.
// ---------------------------------------------------------------------------
namespace imexcl {
constexpr int G = 128, CL = 4, RL = G / CL, H = G / 2, LD = G + 4, LDH = H + 4, LDT = RL + 4;
constexpr int NT = 256, NS = NT / 2;
constexpr int WBUF = (RL + 2) * LD;   // rows -1 .. RL of one species (halo at both ends)
constexpr int TBUF = G * LDT;         // 128 rows of 32 (+4) of one species
constexpr int OFF_CH = 0;                     // Ch[k < H][m], ld LD
constexpr int OFF_CL = OFF_CH + H * LD;       // Cl[m][y < H], ld LDH
constexpr int OFF_MU = OFF_CL + G * LDH;      // mu in the permuted order
constexpr int OFF_W = OFF_MU + G;             // state, 2 species
constexpr int OFF_XR = OFF_W + 2 * WBUF;      // XT[x][y] (step 1) / R[m][y] (step 4), 2 species
constexpr int OFF_K = OFF_XR + 2 * TBUF;      // K[y][m - 32c], 2 species
constexpr int OFF_Z = OFF_K + 2 * TBUF;       // Z[q][m - 32c], 2 species
constexpr int FLOATS = OFF_Z + 2 * TBUF;
constexpr size_t SMEM = sizeof(float) * FLOATS;
static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
static_assert(OFF_CL % 4 == 0 && OFF_MU % 4 == 0 && OFF_W % 4 == 0 && OFF_XR % 4 == 0 && OFF_K % 4 == 0 &&
                  OFF_Z % 4 == 0 && WBUF % 4 == 0 && TBUF % 4 == 0,
              "float4 alignment of every buffer");
}  // namespace imexcl

// dt F of the four nodes (local row y, x..x+3) of both species, stored
// x-major into XTu, XTv ([x][y], ld LDT); W rows are offset by the halo row.
// ns / ss: the north / south neighbour is the node itself (grid edge).
template <int MODEL>
__device__ __forceinline__ void cl_incr4(const float *__restrict__ Wu, const float *__restrict__ Wv,
                                         float *__restrict__ XTu, float *__restrict__ XTv, int y, int x, bool ns,
                                         bool ss, const CoefF &cf) {
    using namespace imexcl;
    const int o = (y + 1) * LD + x, on = ns ? o : o - LD, os = ss ? o : o + LD;
    float su[4], sv[4], cu[4], cv[4];
    {
        const float4 c = *reinterpret_cast<const float4 *>(Wu + o);
        const float4 n = *reinterpret_cast<const float4 *>(Wu + on);
        const float4 s = *reinterpret_cast<const float4 *>(Wu + os);
        const float w = x > 0 ? Wu[o - 1] : c.x, e = x + 4 < G ? Wu[o + 4] : c.w;
        cu[0] = c.x; cu[1] = c.y; cu[2] = c.z; cu[3] = c.w;
        su[0] = (n.x + s.x) + (w + c.y);
        su[1] = (n.y + s.y) + (c.x + c.z);
        su[2] = (n.z + s.z) + (c.y + c.w);
        su[3] = (n.w + s.w) + (c.z + e);
    }
    {
        const float4 c = *reinterpret_cast<const float4 *>(Wv + o);
        const float4 n = *reinterpret_cast<const float4 *>(Wv + on);
        const float4 s = *reinterpret_cast<const float4 *>(Wv + os);
        const float w = x > 0 ? Wv[o - 1] : c.x, e = x + 4 < G ? Wv[o + 4] : c.w;
        cv[0] = c.x; cv[1] = c.y; cv[2] = c.z; cv[3] = c.w;
        sv[0] = (n.x + s.x) + (w + c.y);
        sv[1] = (n.y + s.y) + (c.x + c.z);
        sv[2] = (n.z + s.z) + (c.y + c.w);
        sv[3] = (n.w + s.w) + (c.z + e);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float du, dv;
        incr<MODEL>(cu[j], cv[j], su[j], sv[j], cf, du, dv);
        XTu[(x + j) * LDT + y] = du;
        XTv[(x + j) * LDT + y] = dv;
    }
}

// Forward half-length product over the k-major operand IN (ld LDT, 128
// rows): acc[i][j] = sum_{k<H} Ch[k][s_i] (IN[k][4b + j] +- IN[G-1-k][4b + j])
// with s_i = 4a + i (even part, +) and H + 4a + i - 4 (i >= 4, odd part, -).
__device__ __forceinline__ void cl_fwd(const float *__restrict__ Ch, const float *__restrict__ IN, int a, int b,
                                       float (&acc)[8][4]) {
    using namespace imexcl;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 16
    for (int k = 0; k < H; ++k) {
        float ae[4], ao[4], y1[4], y2[4];
        f4a(ae, *reinterpret_cast<const float4 *>(Ch + k * LD + 4 * a));
        f4a(ao, *reinterpret_cast<const float4 *>(Ch + k * LD + 4 * a + H));
        f4a(y1, *reinterpret_cast<const float4 *>(IN + k * LDT + 4 * b));
        f4a(y2, *reinterpret_cast<const float4 *>(IN + (G - 1 - k) * LDT + 4 * b));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float e = y1[j] + y2[j], o = y1[j] - y2[j];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][j] = fmaf(ae[i], e, acc[i][j]);
                acc[4 + i][j] = fmaf(ao[i], o, acc[4 + i][j]);
            }
        }
    }
}

// Inverse half sums: E[i][j] = sum_{k<H} A[k][4a + i] B[k][4b + j],
// O[i][j] = sum_{k<H} A[k + H][4a + i] B[k + H][4b + j].
template <int LDA, int LDB>
__device__ __forceinline__ void cl_inv(const float *__restrict__ A, const float *__restrict__ B, int a, int b,
                                       float (&E)[4][4], float (&O)[4][4]) {
    using namespace imexcl;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) E[i][j] = O[i][j] = 0.f;
#pragma unroll 16
    for (int k = 0; k < H; ++k) {
        float a1[4], a2[4], b1[4], b2[4];
        f4a(a1, *reinterpret_cast<const float4 *>(A + k * LDA + 4 * a));
        f4a(a2, *reinterpret_cast<const float4 *>(A + (k + H) * LDA + 4 * a));
        f4a(b1, *reinterpret_cast<const float4 *>(B + k * LDB + 4 * b));
        f4a(b2, *reinterpret_cast<const float4 *>(B + (k + H) * LDB + 4 * b));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                E[i][j] = fmaf(a1[i], b1[j], E[i][j]);
                O[i][j] = fmaf(a2[i], b2[j], O[i][j]);
            }
    }
}

template <int MODEL>
__global__ void __launch_bounds__(imexcl::NT, 1)
rd_imex_cl_kernel(float *__restrict__ fields, int64_t field_offset, CoefF cf, float a_u, float a_v,
                  const float *__restrict__ tab, int64_t steps, double p0, double p1, double p2, double p3,
                  double *__restrict__ residual, uint32_t *__restrict__ status) {
    using namespace imexcl;
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) float sm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int cr = (int)cluster.block_rank();
    const int tid = threadIdx.x, r = blockIdx.x / CL;
    float *sCh = sm + OFF_CH, *sCl = sm + OFF_CL, *sMu = sm + OFF_MU, *sW = sm + OFF_W, *sXR = sm + OFF_XR,
          *sK = sm + OFF_K, *sZ = sm + OFF_Z;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;
    const int y0 = cr * RL;

    // tables (Ch: H rows of G, Cl: G rows of H, mu: G)
    for (int q = threadIdx.x; q < H * (G / 4); q += NT) {
        const int y = q / (G / 4), x = (q - y * (G / 4)) * 4;
        *reinterpret_cast<float4 *>(sCh + y * LD + x) = *reinterpret_cast<const float4 *>(tab + y * G + x);
    }
    for (int q = threadIdx.x; q < G * (H / 4); q += NT) {
        const int y = q / (H / 4), x = (q - y * (H / 4)) * 4;
        *reinterpret_cast<float4 *>(sCl + y * LDH + x) = *reinterpret_cast<const float4 *>(tab + H * G + y * H + x);
    }
    for (int q = threadIdx.x; q < G; q += NT) sMu[q] = tab[2 * H * G + q];
    // own rows and the two halo rows that exist, in the state form
    for (int q = threadIdx.x; q < (RL + 2) * (G / 4); q += NT) {
        const int yl = q / (G / 4) - 1, x = (q % (G / 4)) * 4, yg = y0 + yl;
        if (yg < 0 || yg >= G) continue;
        float4 u = *reinterpret_cast<const float4 *>(base + yg * G + x);
        float4 v = *reinterpret_cast<const float4 *>(base + G * G + yg * G + x);
        to_state<MODEL>(u.x, v.x, cf);
        to_state<MODEL>(u.y, v.y, cf);
        to_state<MODEL>(u.z, v.z, cf);
        to_state<MODEL>(u.w, v.w, cf);
        *reinterpret_cast<float4 *>(sW + (yl + 1) * LD + x) = u;
        *reinterpret_cast<float4 *>(sW + WBUF + (yl + 1) * LD + x) = v;
    }
    __syncthreads();

    const int sp = tid / NS, l = tid - sp * NS;
    // products of steps 2-4: a = spectral / row quad (0..15), b = column quad (0..7)
    const int a = l >> 3, b = l & 7;
    // step 5: a5 = local row quad (0..7), b5 = x quad (0..15)
    const int a5 = l >> 4, b5 = l & 15;
    float *XR = sXR + sp * TBUF, *K = sK + sp * TBUF, *Z = sZ + sp * TBUF, *W = sW + sp * WBUF;
    // destinations in the other CTAs (this species' buffers)
    float *k_even = cluster.map_shared_rank(K, a >> 3), *k_odd = cluster.map_shared_rank(K, 2 + (a >> 3));
    float *r_lo = cluster.map_shared_rank(XR, a >> 3), *r_hi = cluster.map_shared_rank(XR, 3 - (a >> 3));
    float *w_up = cr > 0 ? cluster.map_shared_rank(W, cr - 1) : nullptr;
    float *w_dn = cr < CL - 1 ? cluster.map_shared_rank(W, cr + 1) : nullptr;
    // divisors of this thread's step-3 outputs: 1 / (1 + a_s (mu_q + mu_m))
    float dv[8][4];
    {
        const float as = sp ? a_v : a_u;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = (i < 4 ? 4 * a + i : H + 4 * a + i - 4), m = y0 + 4 * b + j;
                dv[i][j] = 1.f / fmaf(as, sMu[q] + sMu[m], 1.f);
            }
    }

    for (int64_t n = 0; n < steps; ++n) {
        // the neighbours' edge rows of the previous step are in place
        cluster.sync();
        // 1. dt F(w^n), x-major
        for (int q = tid; q < RL * (G / 4); q += NT) {
            const int y = q % RL, x = (q / RL) * 4;
            cl_incr4<MODEL>(sW, sW + WBUF, sXR, sXR + TBUF, y, x, cr == 0 && y == 0, cr == CL - 1 && y == RL - 1,
                            cf);
        }
        __syncthreads();
        // 2. forward along x: Xh[y0 + 4b + j][m], m = 4a + i / H + 4a + i - 4
        {
            float acc[8][4];
            cl_fwd(sCh, XR, a, b, acc);
            const int col = 4 * (a & 7);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int row = (y0 + 4 * b + j) * LDT + col;
                *reinterpret_cast<float4 *>(k_even + row) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
                *reinterpret_cast<float4 *>(k_odd + row) = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
            }
        }
        cluster.sync();
        // 3. forward along y, divisors: Z[q][4b + j]
        {
            float acc[8][4];
            cl_fwd(sCh, K, a, b, acc);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = (i < 4 ? 4 * a + i : H + 4 * a + i - 4);
                *reinterpret_cast<float4 *>(Z + q * LDT + 4 * b) =
                    make_float4(acc[i][0] * dv[i][0], acc[i][1] * dv[i][1], acc[i][2] * dv[i][2],
                                acc[i][3] * dv[i][3]);
            }
        }
        __syncthreads();
        // 4. inverse along y: Yh[y][y0 + 4b + j] for y = 4a + i and G-1-(4a + i),
        //    into R[m][y mod 32] of the row's owner
        {
            float E[4][4], O[4][4];
            cl_inv<LDH, LDT>(sCl, Z, a, b, E, O);
            const int clo = 4 * (a & 7), chi = RL - 4 - 4 * (a & 7);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int row = (y0 + 4 * b + j) * LDT;
                *reinterpret_cast<float4 *>(r_lo + row + clo) = make_float4(
                    E[0][j] + O[0][j], E[1][j] + O[1][j], E[2][j] + O[2][j], E[3][j] + O[3][j]);
                *reinterpret_cast<float4 *>(r_hi + row + chi) = make_float4(
                    E[3][j] - O[3][j], E[2][j] - O[2][j], E[1][j] - O[1][j], E[0][j] - O[0][j]);
            }
        }
        cluster.sync();
        // 5. inverse along x, added to the state (rows 4a5 + i, columns 4b5 + j and G-1-(4b5 + j))
        {
            float E[4][4], O[4][4];
            cl_inv<LDT, LDH>(XR, sCl, a5, b5, E, O);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int yl = 4 * a5 + i, o = (yl + 1) * LD;
                float4 lo = *reinterpret_cast<const float4 *>(W + o + 4 * b5);
                lo.x += E[i][0] + O[i][0]; lo.y += E[i][1] + O[i][1]; lo.z += E[i][2] + O[i][2];
                lo.w += E[i][3] + O[i][3];
                *reinterpret_cast<float4 *>(W + o + 4 * b5) = lo;
                float4 hi = *reinterpret_cast<const float4 *>(W + o + G - 4 - 4 * b5);
                hi.x += E[i][3] - O[i][3]; hi.y += E[i][2] - O[i][2]; hi.z += E[i][1] - O[i][1];
                hi.w += E[i][0] - O[i][0];
                *reinterpret_cast<float4 *>(W + o + G - 4 - 4 * b5) = hi;
                if (yl == 0 && w_up) {   // the upper neighbour's bottom halo row
                    *reinterpret_cast<float4 *>(w_up + (RL + 1) * LD + 4 * b5) = lo;
                    *reinterpret_cast<float4 *>(w_up + (RL + 1) * LD + G - 4 - 4 * b5) = hi;
                }
                if (yl == RL - 1 && w_dn) {   // the lower neighbour's top halo row
                    *reinterpret_cast<float4 *>(w_dn + 4 * b5) = lo;
                    *reinterpret_cast<float4 *>(w_dn + G - 4 - 4 * b5) = hi;
                }
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < RL * (G / 4); q += NT) {
        const int yl = q / (G / 4), x = (q - yl * (G / 4)) * 4;
        float4 u = *reinterpret_cast<const float4 *>(sW + (yl + 1) * LD + x);
        float4 v = *reinterpret_cast<const float4 *>(sW + WBUF + (yl + 1) * LD + x);
        from_state<MODEL>(u.x, v.x, cf);
        from_state<MODEL>(u.y, v.y, cf);
        from_state<MODEL>(u.z, v.z, cf);
        from_state<MODEL>(u.w, v.w, cf);
        *reinterpret_cast<float4 *>(base + (y0 + yl) * G + x) = u;
        *reinterpret_cast<float4 *>(base + G * G + (y0 + yl) * G + x) = v;
    }
    // every CTA's rows stored, and no CTA touches another's shared memory
    // after this barrier
    cluster.sync();
    if (cr != 0) return;
    residual_from_global<MODEL, G>(base, p0, p1, p2, p3, residual, status, r, sCh);
}

// Output tile per thread (TM x TN): 0 = 4 x 4, 1 = 8 x 4, 2 = 4 x 8, 3 = 8 x 8.
// Every tile runs the same FMA chains (k ascending per output), so all give
// bit-identical fields; the choice (per G) is a speed knob.  4 = the
// even/odd split (half the FMAs, its own rounding).
// defaults from FHN x 128 realisations, dt = 2^-6, 300 steps on B300 (us
// per step for 4x4 / 8x4 / 4x8 / 8x8 / even-odd): G = 64: 16.8 / 15.0 /
// 15.0 / 16.8 / 10.4 (9.1 once its k-loops were fully unrolled); G = 32:
// 4.67 / 6.04 / 6.13 / 9.32 / 4.09
static int g_imex_var[2] = {4, 4};   // [G == 64]

int imex_n_variants() { return 5; }
bool imex_set_variant(int G, int v) {
    if ((G != 32 && G != 64) || v < 0 || v > 4) return false;
    g_imex_var[G == 64] = v;
    return true;
}
int imex_get_variant(int G) { return (G == 32 || G == 64) ? g_imex_var[G == 64] : -1; }

// floats of the even/odd table at G
size_t imex_eo_table_floats(int G) { return (size_t)G * G + G; }

// both tables of grid side G, into memory the handle owns (rd_init)
rd_status imex_tables_fill(int G, float *tab, float *eo_tab, cudaStream_t s) {
    if (tab) {
        imex_table_kernel<<<(G * G + 127) / 128, 128, 0, s>>>(G, tab);
        note_launch();
    }
    imex_eo_table_kernel<<<(G * G / 2 + 127) / 128, 128, 0, s>>>(G, eo_tab);
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL, int G>
static rd_status launch_imex_eo(const GroupDev &g, const float *tab, float *fields, double *residual,
                                uint32_t *status, cudaStream_t s) {
    constexpr size_t smem = imex_eo_smem<G>();
    auto kern = rd_imex_eo_kernel<MODEL, G>;
    RD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const double h2 = (double)(g.G - 1) * (double)(g.G - 1);
    const float a_u = (float)(g.dt * g.p[0] * h2), a_v = (float)(g.dt * g.p[1] * h2);
    kern<<<g.n_real, G * G / 16, smem, s>>>(fields, g.field_offset, make_coef(g), a_u, a_v, tab, g.n_steps,
                                            g.p[0], g.p[1], g.p[2], g.p[3],
                                            residual ? residual + 2 * g.real_base : nullptr, status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL, int G, int TM, int TN>
static rd_status launch_imex_mgt(const GroupDev &g, float *fields, const float *tab, double *residual,
                                 uint32_t *status, cudaStream_t s) {
    constexpr size_t smem = imex_smem<G>();
    auto kern = rd_imex_kernel<MODEL, G, TM, TN>;
    RD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const double h2 = (double)(g.G - 1) * (double)(g.G - 1);
    const float a_u = (float)(g.dt * g.p[0] * h2), a_v = (float)(g.dt * g.p[1] * h2);
    kern<<<g.n_real, 2 * (G / TM) * (G / TN), smem, s>>>(fields, g.field_offset, make_coef(g), a_u, a_v, tab,
                                                          g.n_steps, g.p[0], g.p[1], g.p[2], g.p[3],
                                                          residual ? residual + 2 * g.real_base : nullptr, status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL, int G>
static rd_status launch_imex_mg(const GroupDev &g, float *fields, const float *tab, const float *eo_tab,
                                double *residual, uint32_t *status, cudaStream_t s) {
    switch (g_imex_var[G == 64]) {
        case 1: return launch_imex_mgt<MODEL, G, 8, 4>(g, fields, tab, residual, status, s);
        case 2: return launch_imex_mgt<MODEL, G, 4, 8>(g, fields, tab, residual, status, s);
        case 3: return launch_imex_mgt<MODEL, G, 8, 8>(g, fields, tab, residual, status, s);
        case 4: return launch_imex_eo<MODEL, G>(g, eo_tab, fields, residual, status, s);
        default: return launch_imex_mgt<MODEL, G, 4, 4>(g, fields, tab, residual, status, s);
    }
}

template <int G>
static rd_status launch_imex_g(const GroupDev &g, float *fields, const float *tab, const float *eo_tab,
                               double *residual, uint32_t *status, cudaStream_t s) {
    switch (g.model) {
        case RD_FHN: return launch_imex_mg<RD_FHN, G>(g, fields, tab, eo_tab, residual, status, s);
        case RD_GM: return launch_imex_mg<RD_GM, G>(g, fields, tab, eo_tab, residual, status, s);
        case RD_DIFF: return launch_imex_mg<RD_DIFF, G>(g, fields, tab, eo_tab, residual, status, s);
        case RD_BZ: return launch_imex_mg<RD_BZ, G>(g, fields, tab, eo_tab, residual, status, s);
        default: return RD_ERR_UNSUPPORTED;
    }
}

// G = 128: one cluster of four CTAs per realisation
template <int MODEL>
static rd_status launch_imex_cl_m(const GroupDev &g, const float *eo_tab, float *fields, double *residual,
                                  uint32_t *status, cudaStream_t s) {
    using namespace imexcl;
    auto kern = rd_imex_cl_kernel<MODEL>;
    rd_status st = smem_attr(kern, (int)SMEM);
    if (st) return st;
    const double h2 = (double)(g.G - 1) * (double)(g.G - 1);
    const float a_u = (float)(g.dt * g.p[0] * h2), a_v = (float)(g.dt * g.p[1] * h2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g.n_real * CL), 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    RD_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, fields, g.field_offset, make_coef(g), a_u, a_v, eo_tab, g.n_steps,
                                   g.p[0], g.p[1], g.p[2], g.p[3],
                                   residual ? residual + 2 * g.real_base : nullptr, status));
    note_launch();
    return cuda_status(cudaGetLastError());
}

static rd_status launch_imex_cl(const GroupDev &g, const float *eo_tab, float *fields, double *residual,
                                uint32_t *status, cudaStream_t s) {
    switch (g.model) {
        case RD_FHN: return launch_imex_cl_m<RD_FHN>(g, eo_tab, fields, residual, status, s);
        case RD_GM: return launch_imex_cl_m<RD_GM>(g, eo_tab, fields, residual, status, s);
        case RD_DIFF: return launch_imex_cl_m<RD_DIFF>(g, eo_tab, fields, residual, status, s);
        case RD_BZ: return launch_imex_cl_m<RD_BZ>(g, eo_tab, fields, residual, status, s);
        default: return RD_ERR_UNSUPPORTED;
    }
}

int imex_table_index(int G) { return G == 32 ? 0 : G == 64 ? 1 : G == 128 ? 2 : -1; }

bool imex_supported(const GroupDev &g) {
    return g.model != RD_RDODE && imex_table_index(g.G) >= 0;
}

rd_status launch_imex_group(const GroupDev &g, const float *tab, const float *eo_tab, float *fields, double *residual,
                            uint32_t *status, cudaStream_t s) {
    if (!imex_supported(g) || !eo_tab || (g.G != 128 && !tab)) return RD_ERR_UNSUPPORTED;
    if (g.n_steps == 0 && !residual) return RD_OK;
    if (g.G == 128) return launch_imex_cl(g, eo_tab, fields, residual, status, s);
    return g.G == 32 ? launch_imex_g<32>(g, fields, tab, eo_tab, residual, status, s)
                     : launch_imex_g<64>(g, fields, tab, eo_tab, residual, status, s);
}

}  // namespace rdcil
