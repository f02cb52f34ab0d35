// Register-tile helpers shared by the resident forward stepper and the
// resident adjoint stepper.
//
// A G x G field is split into TY x TX tiles, one per thread: NX = G/TX
// threads along x (a power of two <= 32, so a warp holds whole tile rows and
// the east/west neighbours of a tile edge are shuffle lanes), NY = G/TY
// along y.  North/south tile edges go through a double-buffered shared
// memory ring halo[buf 2][species 2][edge 2][NY][G] (one barrier per step).
// (Extra ring slots holding the mirror ghosts, which make the north/south
// reads unconditional, measured 9 % slower on FHN 64x64: the edge tiles'
// extra stores cost more than the tests they remove.)
#pragma once
#include "common.cuh"

namespace rdcil {

template <int G, int TY, int TX>
struct Tiling {
    static constexpr int NX = G / TX;
    static constexpr int NY = G / TY;
    static constexpr int NT = NX * NY;
    static constexpr int HALO_FLOATS = 2 * 2 * 2 * NY * G;
    static constexpr size_t SMEM = (size_t)HALO_FLOATS * sizeof(float);
    static_assert(NX <= 32 && (NX & (NX - 1)) == 0, "tile row must fit a warp");
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
};

template <int TX>
__device__ __forceinline__ void st_row(float *dst, const float (&a)[TX]) {
    if constexpr (TX % 4 == 0) {
#pragma unroll
        for (int c = 0; c < TX; c += 4)
            *reinterpret_cast<float4 *>(dst + c) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
    } else if constexpr (TX == 2) {
        *reinterpret_cast<float2 *>(dst) = make_float2(a[0], a[1]);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) dst[c] = a[c];
    }
}

template <int TX>
__device__ __forceinline__ void ld_row(const float *src, float (&a)[TX]) {
    if constexpr (TX % 4 == 0) {
#pragma unroll
        for (int c = 0; c < TX; c += 4) {
            float4 t = *reinterpret_cast<const float4 *>(src + c);
            a[c] = t.x; a[c + 1] = t.y; a[c + 2] = t.z; a[c + 3] = t.w;
        }
    } else if constexpr (TX == 2) {
        float2 t = *reinterpret_cast<const float2 *>(src);
        a[0] = t.x; a[1] = t.y;
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) a[c] = src[c];
    }
}

template <int G, int TY, int TX>
__device__ __forceinline__ void halo_put(float *hb, int tx, int ty, const float (&u)[TY][TX],
                                         const float (&v)[TY][TX]) {
    constexpr int NY = Tiling<G, TY, TX>::NY;
    const int x0 = tx * TX;
    st_row<TX>(hb + ((0 * 2 + 0) * NY + ty) * G + x0, u[0]);
    st_row<TX>(hb + ((0 * 2 + 1) * NY + ty) * G + x0, u[TY - 1]);
    st_row<TX>(hb + ((1 * 2 + 0) * NY + ty) * G + x0, v[0]);
    st_row<TX>(hb + ((1 * 2 + 1) * NY + ty) * G + x0, v[TY - 1]);
}

// North neighbour row of the tile's first row (mirror ghost at the top edge).
template <int G, int TY, int TX>
__device__ __forceinline__ void halo_north(const float *hb, int tx, int ty, const float (&u)[TY][TX],
                                           const float (&v)[TY][TX], float (&pu)[TX], float (&pv)[TX]) {
    constexpr int NY = Tiling<G, TY, TX>::NY;
    const int x0 = tx * TX;
    if (ty > 0) {
        ld_row<TX>(hb + ((0 * 2 + 1) * NY + ty - 1) * G + x0, pu);
        ld_row<TX>(hb + ((1 * 2 + 1) * NY + ty - 1) * G + x0, pv);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) { pu[c] = u[0][c]; pv[c] = v[0][c]; }
    }
}

// South neighbour row of tile row i (inside the tile, from the halo, or the
// mirror ghost at the bottom edge).
template <int G, int TY, int TX>
__device__ __forceinline__ void row_south(const float *hb, int tx, int ty, int i, const float (&u)[TY][TX],
                                          const float (&v)[TY][TX], float (&su)[TX], float (&sv)[TX]) {
    constexpr int NY = Tiling<G, TY, TX>::NY;
    const int x0 = tx * TX;
    if (i + 1 < TY) {
#pragma unroll
        for (int c = 0; c < TX; ++c) { su[c] = u[i + 1][c]; sv[c] = v[i + 1][c]; }
    } else if (ty < NY - 1) {
        ld_row<TX>(hb + ((0 * 2 + 0) * NY + ty + 1) * G + x0, su);
        ld_row<TX>(hb + ((1 * 2 + 0) * NY + ty + 1) * G + x0, sv);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) { su[c] = u[TY - 1][c]; sv[c] = v[TY - 1][c]; }
    }
}

// West/east neighbours of the first/last cell of a tile row (shuffle lanes,
// mirror ghost at the domain edge).  Every lane of the warp must call this.
template <int NX>
__device__ __forceinline__ void row_west_east(int tx, float first, float last, float &w, float &e) {
    w = __shfl_up_sync(0xffffffffu, last, 1, NX);
    e = __shfl_down_sync(0xffffffffu, first, 1, NX);
    if (tx == 0) w = first;
    if (tx == NX - 1) e = last;
}

// FP32 kinetics with coefficients folded with dt and (G-1)^2 on the host:
//   cu = Du dt (G-1)^2, cv = Dv dt (G-1)^2, k1 = dt,
//   FHN: k2 = eps dt, k3 = a;   GM: k2 = rho dt, k3 = mu;   BZ: k3 = B.
// GM is stepped in deviation form (see euler_cell): u0, v0 = the FP32
// equilibrium (1/mu, 1/mu^2), tu0 = 2 u0, e0 = u0 - mu v0 and e1 = u0^2 - v0
// (evaluated in FP64, rounded once; both are 0 when 1/mu is exact).
// The v update folds the node's own weight with the -4 of the 5-point
// stencil (FP64 on the host, rounded once):
//   FHN: be = 1 - 4 cv - k2 k3;   GM: be = 1 - 4 cv - k2, k2e1 = k2 e1.
// (v relaxes quickly, so the rounding of be does not accumulate; u keeps
// the form u + increments, because a rounded weight near 1 on u itself
// would bias every step the same way.)
// BZ (Brusselator) is stepped in deviation form too: u0 = A, v0 = the FP32
// B/A, and with a = u - u0, b = v - v0, P = v0 a^2 + (u0 + a)^2 b:
//   f = e0 + c1 a + P,   g = -e0 + c2 a - P,
//   e0 = A (A v0 - B), c1 = 2 A v0 - (B + 1), c2 = B - 2 A v0   (FP64, rounded once)
// (exact in real arithmetic; e0 = 0 and c1 = B - 1, c2 = -B when B/A is exact).
struct CoefF {
    float cu, cv, k1, k2, k3;
    float u0, v0, tu0, e0, e1;
    float be, k2e1;
    float c1, c2;
};

inline CoefF make_coef(const GroupDev &g) {
    double g1 = (double)(g.G - 1);
    double h2 = g1 * g1;
    CoefF c{};
    const double cu = g.p[0] * g.dt * h2, cv = g.p[1] * g.dt * h2;
    c.cu = (float)cu;
    c.cv = (float)cv;
    c.k1 = (float)g.dt;
    if (g.model == RD_FHN || g.model == RD_GM || g.model == RD_BZ) {
        c.k2 = (float)(g.p[2] * g.dt);
        c.k3 = (float)g.p[3];
    }
    if (g.model == RD_FHN) c.be = (float)(1.0 - 4.0 * cv - g.p[2] * g.dt * g.p[3]);
    if (g.model == RD_BZ) {
        const double A = g.p[2], B = g.p[3];
        const float v0 = (float)(B / A);
        c.u0 = (float)A;
        c.v0 = v0;
        c.e0 = (float)(A * (A * (double)v0 - B));
        c.c1 = (float)(2.0 * A * (double)v0 - (B + 1.0));
        c.c2 = (float)(B - 2.0 * A * (double)v0);
    }
    if (g.model == RD_GM) {
        double mu = g.p[3], k2 = g.p[2] * g.dt;
        float u0 = (float)(1.0 / mu);
        float v0 = (float)((double)u0 * (double)u0);
        c.u0 = u0;
        c.v0 = v0;
        c.tu0 = 2.0f * u0;
        const double e0 = (double)u0 - mu * (double)v0, e1 = (double)u0 * (double)u0 - (double)v0;
        c.e0 = (float)e0;
        c.e1 = (float)e1;
        c.be = (float)(1.0 - 4.0 * cv - k2);
        c.k2e1 = (float)(k2 * e1);
    }
    return c;
}

// State registers hold (u, v) for FHN and DIFF, and the deviation (a, b) =
// (u - u0, v - v0) from the FP32 equilibrium for GM.  These convert.
template <int MODEL>
__device__ __forceinline__ void to_state(float &u, float &v, const CoefF &c) {
    if (MODEL == RD_GM || MODEL == RD_BZ) { u -= c.u0; v -= c.v0; }
}
template <int MODEL>
__device__ __forceinline__ void from_state(float &u, float &v, const CoefF &c) {
    if (MODEL == RD_GM || MODEL == RD_BZ) { u += c.u0; v += c.v0; }
}

// x / y for the GM kinetics: x times the hardware approximate reciprocal of
// y (PTX rcp.approx.ftz.f32; the ISA bounds its error by one unit in the
// last place, subnormals flushed).  y is the inhibitor concentration, about
// 1/mu^2, far from both ends of the FP32 range.  Every explicit GM stepper
// path uses it, so they stay bit-identical to one another; the FP32 field
// tolerance against the FP64 oracle covers its rounding.
__device__ __forceinline__ float quot_fast(float x, float y) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return x * r;
}

// One explicit Euler update of a node given the neighbour sums
// su = (N + S) + (W + E) of both species (of the state registers; the
// Laplacian of a deviation equals that of the field):
//   FHN: u' = u + cu (su - 4u) + k1 (u - u^3 - v),   v' = be v + k2 u + cv sv
// (= v + dt (Dv Lap v + eps (u - a v)) with the folded weight be).
template <int MODEL>
__device__ __forceinline__ void euler_cell(float u, float v, float su, float sv, const CoefF &c, float &un,
                                           float &vn) {
    if (MODEL == RD_FHN) {
        float ru = fmaf(-u * u, u, u - v);
        un = fmaf(c.cu, fmaf(-4.f, u, su), fmaf(c.k1, ru, u));
        vn = fmaf(c.be, v, fmaf(c.k2, u, c.cv * sv));
    } else if (MODEL == RD_GM) {
        // Deviation form, exact in real arithmetic for U = u0 + a, V = v0 + b:
        //   U^2/V - mu U = U (a - mu b + e0) / V,   U^2 - V = a (2 u0 + a) - b + e1
        // so the increments carry the relative precision of the deviation
        // rather than of the equilibrium value:
        //   a' = a + cu (sa - 4a) + k2 U (a - mu b + e0) / V
        //   b' = be b + cv sb + k2 a (a + 2 u0) + k2 e1
        const float a = u, b = v;
        float U = a + c.u0, V = b + c.v0;
        float t = fmaf(-c.k3, b, a + c.e0);
        float f = quot_fast(U * t, V);
        un = fmaf(c.cu, fmaf(-4.f, a, su), fmaf(c.k2, f, a));
        vn = fmaf(c.be, b, fmaf(c.k2 * a, a + c.tu0, fmaf(c.cv, sv, c.k2e1)));
    } else if (MODEL == RD_BZ) {
        // deviation form (see CoefF): f = e0 + c1 a + P, g = -e0 + c2 a - P
        const float a = u, b = v;
        const float U = a + c.u0;
        const float P = fmaf(c.v0 * a, a, (U * U) * b);
        const float f = fmaf(c.c1, a, c.e0 + P);
        const float g = fmaf(c.c2, a, -c.e0 - P);
        un = fmaf(c.cu, fmaf(-4.f, a, su), fmaf(c.k1, f, a));
        vn = fmaf(c.cv, fmaf(-4.f, b, sv), fmaf(c.k1, g, b));
    } else {
        un = fmaf(c.cu, fmaf(-4.f, u, su), u);
        vn = fmaf(c.cv, fmaf(-4.f, v, sv), v);
    }
}

// FP64 right-hand side at one node from FP32 neighbours (used for the
// residual; operation order of the plain definition).
template <int MODEL>
__device__ __forceinline__ void rhs_f64(double u, double v, double nu, double su, double wu, double eu,
                                        double nv, double sv, double wv, double ev, const double *p,
                                        double h2, double &Fu, double &Fv) {
    double lu = ((((eu + wu) + su) + nu) - 4.0 * u) * h2;
    double lv = ((((ev + wv) + sv) + nv) - 4.0 * v) * h2;
    double ru, rv;
    if (MODEL == RD_FHN) {
        ru = (u - (u * u) * u) - v;
        rv = p[2] * (u - p[3] * v);
    } else if (MODEL == RD_GM) {
        double uu = u * u;
        ru = p[2] * (uu / v - p[3] * u);
        rv = p[2] * (uu - v);
    } else if (MODEL == RD_BZ) {
        double uuv = (u * u) * v;
        ru = (p[2] - (p[3] + 1.0) * u) + uuv;
        rv = p[3] * u - uuv;
    } else {
        ru = 0.0;
        rv = 0.0;
    }
    Fu = p[0] * lu + ru;
    Fv = p[1] * lv + rv;
}

// Barrier policies for code that one group of threads runs on one
// realisation: the whole CTA (barrier 0), or one half of a 512-thread CTA
// (named barrier 1 + h over its 256 threads, so the two halves integrate
// two realisations independently).
struct SyncAll {
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ int nthreads() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int sync_or(int p) const { return __syncthreads_or(p); }
};
struct SyncHalf {
    int h;   // 0 or 1
    __device__ __forceinline__ int tid() const { return threadIdx.x & 255; }
    __device__ __forceinline__ int nthreads() const { return 256; }
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync %0, 256;" ::"r"(1 + h) : "memory");
    }
    __device__ __forceinline__ int sync_or(int p) const {
        int r;
        asm volatile(
            "{\n\t.reg .pred q, o;\n\t"
            "setp.ne.s32 q, %1, 0;\n\t"
            "bar.red.or.pred o, %2, 256, q;\n\t"
            "selp.s32 %0, 1, 0, o;\n\t}"
            : "=r"(r)
            : "r"(p), "r"(1 + h)
            : "memory");
        return r;
    }
};

// FP64 steady-state residual of the final state of realisation r, read
// back from global memory after the block stored it (block-visible after
// the barrier): max |F| and sqrt(mean F^2) over both species, F from the
// stored FP32 values in the plain operation order.  Thread t takes nodes
// t, t + NT, ...; the sum is reduced with warp shuffles, then across warps.
// sy: the threads that integrate this realisation (barrier policy above).
template <int MODEL, int G, class Sync = SyncAll>
__device__ __forceinline__ void residual_from_global(const float *__restrict__ base, double p0, double p1, double p2,
                                                     double p3, double *__restrict__ residual,
                                                     uint32_t *__restrict__ status, int r, void *smem,
                                                     Sync sy = Sync{}) {
    sy.sync();
    const double p[4] = {p0, p1, p2, p3};
    const double h2 = (double)(G - 1) * (double)(G - 1);
    const float *u = base, *v = base + G * G;
    const int tid = sy.tid(), nt = sy.nthreads();
    double mx = 0.0, ss = 0.0;
    bool bad = false;
    for (int k = tid; k < G * G; k += nt) {
        const int y = k / G, x = k - y * G;
        const int kn = (y > 0 ? k - G : k), ks = (y < G - 1 ? k + G : k);
        const int kw = (x > 0 ? k - 1 : k), ke = (x < G - 1 ? k + 1 : k);
        double Fu, Fv;
        rhs_f64<MODEL>(u[k], v[k], u[kn], u[ks], u[kw], u[ke], v[kn], v[ks], v[kw], v[ke], p, h2, Fu, Fv);
        bad |= !isfinite(u[k]) || !isfinite(v[k]) || !isfinite(Fu) || !isfinite(Fv);
        mx = fmax(mx, fmax(fabs(Fu), fabs(Fv)));
        ss += Fu * Fu + Fv * Fv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    const int anybad = sy.sync_or(bad ? 1 : 0);
    double *red = reinterpret_cast<double *>(smem);
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    if (lane == 0) { red[warp] = mx; red[nw + warp] = ss; }
    sy.sync();
    if (tid == 0) {
        double m = 0.0, s = 0.0;
        for (int wi = 0; wi < nw; ++wi) { m = fmax(m, red[wi]); s += red[nw + wi]; }
        if (anybad) {
            atomicOr(status, (unsigned)ST_NONFINITE);
            m = __longlong_as_double(0x7ff8000000000000ll);
            s = m;
        }
        if (residual) {
            residual[2 * r] = m;
            residual[2 * r + 1] = sqrt(s / (double)(2 * G * G));
        }
    }
    sy.sync();
}

template <int MODEL, int TY, int TX>
__device__ __forceinline__ void tile_to_state(float (&u)[TY][TX], float (&v)[TY][TX], const CoefF &c) {
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int j = 0; j < TX; ++j) to_state<MODEL>(u[i][j], v[i][j], c);
}
template <int MODEL, int TY, int TX>
__device__ __forceinline__ void tile_from_state(float (&u)[TY][TX], float (&v)[TY][TX], const CoefF &c) {
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int j = 0; j < TX; ++j) from_state<MODEL>(u[i][j], v[i][j], c);
}

template <int G, int TY, int TX>
__device__ __forceinline__ void tile_load(const float *base, int tx, int ty, float (&u)[TY][TX], float (&v)[TY][TX]) {
    const int x0 = tx * TX, y0 = ty * TY;
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        ld_row<TX>(base + (y0 + i) * G + x0, u[i]);
        ld_row<TX>(base + G * G + (y0 + i) * G + x0, v[i]);
    }
}

template <int G, int TY, int TX>
__device__ __forceinline__ void tile_store(float *base, int tx, int ty, const float (&u)[TY][TX],
                                           const float (&v)[TY][TX]) {
    const int x0 = tx * TX, y0 = ty * TY;
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        st_row<TX>(base + (y0 + i) * G + x0, u[i]);
        st_row<TX>(base + G * G + (y0 + i) * G + x0, v[i]);
    }
}

// ---------------------------------------------------------------------------
// Serpentine tiles for the forward stepper.  Lanes with even tx hold their
// tile columns in reverse order (register c = column x0 + TX-1-c), lanes
// with odd tx in natural order.  Then across the boundary between tx = 2k
// and 2k+1 both lanes hold the boundary column in register 0, and across
// the boundary between 2k+1 and 2k+2 both hold it in register TX-1: one
// xor-shuffle of register 0 and one indexed shuffle of register TX-1 (the
// source lane fixed for the whole run) give every lane both outside
// neighbours.  A lane at the domain edge names itself as the source and so
// receives its own edge column, which is the mirror ghost.  The Laplacian
// needs only W + E, which does not depend on the column order (addition
// is commutative), so every node's arithmetic is the same as in the
// natural-order tiles of the packed and adjoint kernels.
// Vertically adjacent tiles share tx and so share the column order, which
// keeps the north/south halo ring in register order.
// ---------------------------------------------------------------------------
template <int NX>
__device__ __forceinline__ int serp_src(int tx) {
    const int lane = threadIdx.x & 31;
    if (tx & 1) return tx == NX - 1 ? lane : lane + 1;
    return tx == 0 ? lane : lane - 1;
}

template <int G, int TY, int TX>
__device__ __forceinline__ void tile_load_s(const float *base, int tx, int ty, float (&u)[TY][TX],
                                            float (&v)[TY][TX]) {
    float a[TY][TX], b[TY][TX];
    tile_load<G, TY, TX>(base, tx, ty, a, b);
    const bool rev = !(tx & 1);
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            u[i][c] = rev ? a[i][TX - 1 - c] : a[i][c];
            v[i][c] = rev ? b[i][TX - 1 - c] : b[i][c];
        }
}

template <int G, int TY, int TX>
__device__ __forceinline__ void tile_store_s(float *base, int tx, int ty, const float (&u)[TY][TX],
                                             const float (&v)[TY][TX]) {
    float a[TY][TX], b[TY][TX];
    const bool rev = !(tx & 1);
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            a[i][c] = rev ? u[i][TX - 1 - c] : u[i][c];
            b[i][c] = rev ? v[i][TX - 1 - c] : v[i][c];
        }
    tile_store<G, TY, TX>(base, tx, ty, a, b);
}

// One Euler step of a serpentine tile (reads halo buffer hb after the
// barrier that follows halo_put; mirror ghosts at the top/bottom edge).  (A second, test-free copy of this body for the
// warps away from the top and bottom edges measured 29 % slower on FHN
// 64x64: two unrolled bodies in one loop cost more than the tests.)
template <int MODEL, int G, int TY, int TX>
__device__ __forceinline__ void tile_step_s(const float *hb, int tx, int ty, int src, float (&u)[TY][TX],
                                            float (&v)[TY][TX], const CoefF &cf) {
    float pu[TX], pv[TX];
    halo_north<G, TY, TX>(hb, tx, ty, u, v, pu, pv);
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        float su[TX], sv[TX];
        row_south<G, TY, TX>(hb, tx, ty, i, u, v, su, sv);
        const float xu0 = __shfl_xor_sync(0xffffffffu, u[i][0], 1);
        const float xv0 = __shfl_xor_sync(0xffffffffu, v[i][0], 1);
        const float xu1 = __shfl_sync(0xffffffffu, u[i][TX - 1], src);
        const float xv1 = __shfl_sync(0xffffffffu, v[i][TX - 1], src);
        float cu_[TX], cv_[TX];
#pragma unroll
        for (int c = 0; c < TX; ++c) { cu_[c] = u[i][c]; cv_[c] = v[i][c]; }
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            float Lu = c > 0 ? cu_[c - 1] : xu0, Ru = c < TX - 1 ? cu_[c + 1] : xu1;
            float Lv = c > 0 ? cv_[c - 1] : xv0, Rv = c < TX - 1 ? cv_[c + 1] : xv1;
            float nu = (pu[c] + su[c]) + (Lu + Ru);
            float nv = (pv[c] + sv[c]) + (Lv + Rv);
            euler_cell<MODEL>(cu_[c], cv_[c], nu, nv, cf, u[i][c], v[i][c]);
        }
#pragma unroll
        for (int c = 0; c < TX; ++c) { pu[c] = cu_[c]; pv[c] = cv_[c]; }
    }
}

// ---------------------------------------------------------------------------
// Rotating serpentine tiles.  Updating a tile in place keeps every old row
// alive until the row below it is done (it is that row's north neighbour),
// which costs a register copy of every node per step.  Here the TY rows live
// in R = TY + 1 row slots: logical row i in slot (i + OFF) mod R, one slot
// free.  New row i is written into the slot of old row i - 1 (the free slot
// for row 0), node by node right after that node's north value was read, so
// nothing is copied; the mapping moves by one slot per step (OFF -> OFF - 1
// mod R) and the caller unrolls R steps so that every slot index is a
// compile-time constant.  Per node the arithmetic and its order are those of
// tile_step_s, so the fields are bit-identical.
// ---------------------------------------------------------------------------
template <int G, int TY, int TX, int OFF>
__device__ __forceinline__ void halo_put_rot(float *hb, int tx, int ty, const float (&u)[TY + 1][TX],
                                             const float (&v)[TY + 1][TX]) {
    constexpr int NY = Tiling<G, TY, TX>::NY, R = TY + 1;
    const int x0 = tx * TX;
    st_row<TX>(hb + ((0 * 2 + 0) * NY + ty) * G + x0, u[OFF % R]);
    st_row<TX>(hb + ((0 * 2 + 1) * NY + ty) * G + x0, u[(TY - 1 + OFF) % R]);
    st_row<TX>(hb + ((1 * 2 + 0) * NY + ty) * G + x0, v[OFF % R]);
    st_row<TX>(hb + ((1 * 2 + 1) * NY + ty) * G + x0, v[(TY - 1 + OFF) % R]);
}

template <int MODEL, int G, int TY, int TX, int OFF>
__device__ __forceinline__ void tile_step_rot(const float *hb, int tx, int ty, int src, float (&u)[TY + 1][TX],
                                              float (&v)[TY + 1][TX], const CoefF &cf) {
    constexpr int NY = Tiling<G, TY, TX>::NY, R = TY + 1;
    const int x0 = tx * TX;
    float nu0[TX], nv0[TX];   // north neighbours of row 0: halo, or the row itself at the top edge
    if (ty > 0) {
        ld_row<TX>(hb + ((0 * 2 + 1) * NY + ty - 1) * G + x0, nu0);
        ld_row<TX>(hb + ((1 * 2 + 1) * NY + ty - 1) * G + x0, nv0);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) { nu0[c] = u[OFF % R][c]; nv0[c] = v[OFF % R][c]; }
    }
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        const int pr = (i + OFF) % R;            // old row i
        const int qr = (i + OFF + R - 1) % R;    // old row i - 1 (free slot for i = 0): receives new row i
        const int sr = (i + 1 + OFF) % R;        // old row i + 1
        float sl_u[TX], sl_v[TX];                // south neighbours of the last row
        if (i == TY - 1) {
            if (ty < NY - 1) {
                ld_row<TX>(hb + ((0 * 2 + 0) * NY + ty + 1) * G + x0, sl_u);
                ld_row<TX>(hb + ((1 * 2 + 0) * NY + ty + 1) * G + x0, sl_v);
            } else {
#pragma unroll
                for (int c = 0; c < TX; ++c) { sl_u[c] = u[pr][c]; sl_v[c] = v[pr][c]; }
            }
        }
        const float xu0 = __shfl_xor_sync(0xffffffffu, u[pr][0], 1);
        const float xv0 = __shfl_xor_sync(0xffffffffu, v[pr][0], 1);
        const float xu1 = __shfl_sync(0xffffffffu, u[pr][TX - 1], src);
        const float xv1 = __shfl_sync(0xffffffffu, v[pr][TX - 1], src);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            const float Nu = i == 0 ? nu0[c] : u[qr][c], Nv = i == 0 ? nv0[c] : v[qr][c];
            const float Su = i == TY - 1 ? sl_u[c] : u[sr][c], Sv = i == TY - 1 ? sl_v[c] : v[sr][c];
            const float Lu = c > 0 ? u[pr][c - 1] : xu0, Ru = c < TX - 1 ? u[pr][c + 1] : xu1;
            const float Lv = c > 0 ? v[pr][c - 1] : xv0, Rv = c < TX - 1 ? v[pr][c + 1] : xv1;
            const float nu = (Nu + Su) + (Lu + Ru);
            const float nv = (Nv + Sv) + (Lv + Rv);
            euler_cell<MODEL>(u[pr][c], v[pr][c], nu, nv, cf, u[qr][c], v[qr][c]);
        }
    }
}

}  // namespace rdcil

// ===========================================================================
// Packed (u, v) tiles for the forward stepper.  Each node's two species sit
// in one float2, so the 5-point sums of both species are single packed FP32
// instructions (add.f32x2 / fma.f32x2 of sm_100-family GPUs) and the halo
// moves are float4 (two nodes) wide.  Halo ring: [buf 2][edge 2][NY][G]
// float2 (edge 0 = tile top row, 1 = tile bottom row).
// ===========================================================================
namespace rdcil {

template <int G, int TY, int TX>
struct Tiling2 {
    static constexpr int NX = G / TX;
    static constexpr int NY = G / TY;
    static constexpr int NT = NX * NY;
    static constexpr int HALO_F2 = 2 * 2 * NY * G;          // float2 entries, both buffers
    static constexpr size_t SMEM = (size_t)HALO_F2 * sizeof(float2);
    static_assert(TX % 2 == 0, "tile width must be even (float4 halo moves)");
    static_assert(NX <= 32 && (NX & (NX - 1)) == 0, "tile row must fit a warp");
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
};

template <int TX>
__device__ __forceinline__ void st_row2(float2 *dst, const float2 (&a)[TX]) {
#pragma unroll
    for (int c = 0; c < TX; c += 2)
        *reinterpret_cast<float4 *>(dst + c) = make_float4(a[c].x, a[c].y, a[c + 1].x, a[c + 1].y);
}

template <int TX>
__device__ __forceinline__ void ld_row2(const float2 *src, float2 (&a)[TX]) {
#pragma unroll
    for (int c = 0; c < TX; c += 2) {
        float4 t = *reinterpret_cast<const float4 *>(src + c);
        a[c] = make_float2(t.x, t.y);
        a[c + 1] = make_float2(t.z, t.w);
    }
}

// global layout is [species][y][x]: load/store one tile row of each species
template <int G, int TX>
__device__ __forceinline__ void ld_row_g(const float *base, int y, int x0, float2 (&a)[TX]) {
#pragma unroll
    for (int c = 0; c < TX; c += 4) {
        if (c + 4 <= TX) {
            float4 u = *reinterpret_cast<const float4 *>(base + y * G + x0 + c);
            float4 v = *reinterpret_cast<const float4 *>(base + G * G + y * G + x0 + c);
            a[c] = make_float2(u.x, v.x); a[c + 1] = make_float2(u.y, v.y);
            a[c + 2] = make_float2(u.z, v.z); a[c + 3] = make_float2(u.w, v.w);
        } else {
            float2 u = *reinterpret_cast<const float2 *>(base + y * G + x0 + c);
            float2 v = *reinterpret_cast<const float2 *>(base + G * G + y * G + x0 + c);
            a[c] = make_float2(u.x, v.x); a[c + 1] = make_float2(u.y, v.y);
        }
    }
}

template <int G, int TX>
__device__ __forceinline__ void st_row_g(float *base, int y, int x0, const float2 (&a)[TX]) {
#pragma unroll
    for (int c = 0; c < TX; c += 4) {
        if (c + 4 <= TX) {
            *reinterpret_cast<float4 *>(base + y * G + x0 + c) = make_float4(a[c].x, a[c + 1].x, a[c + 2].x, a[c + 3].x);
            *reinterpret_cast<float4 *>(base + G * G + y * G + x0 + c) =
                make_float4(a[c].y, a[c + 1].y, a[c + 2].y, a[c + 3].y);
        } else {
            *reinterpret_cast<float2 *>(base + y * G + x0 + c) = make_float2(a[c].x, a[c + 1].x);
            *reinterpret_cast<float2 *>(base + G * G + y * G + x0 + c) = make_float2(a[c].y, a[c + 1].y);
        }
    }
}

template <int G, int TY, int TX>
__device__ __forceinline__ void tile2_load(const float *base, int tx, int ty, float2 (&w)[TY][TX]) {
#pragma unroll
    for (int i = 0; i < TY; ++i) ld_row_g<G, TX>(base, ty * TY + i, tx * TX, w[i]);
}

template <int G, int TY, int TX>
__device__ __forceinline__ void tile2_store(float *base, int tx, int ty, const float2 (&w)[TY][TX]) {
#pragma unroll
    for (int i = 0; i < TY; ++i) st_row_g<G, TX>(base, ty * TY + i, tx * TX, w[i]);
}

template <int MODEL>
__device__ __forceinline__ float2 to_state2(float2 w, const CoefF &c) {
    if (MODEL == RD_GM || MODEL == RD_BZ) return __fadd2_rn(w, make_float2(-c.u0, -c.v0));
    return w;
}
template <int MODEL>
__device__ __forceinline__ float2 from_state2(float2 w, const CoefF &c) {
    if (MODEL == RD_GM || MODEL == RD_BZ) return __fadd2_rn(w, make_float2(c.u0, c.v0));
    return w;
}

// One Euler update of a node: C = (u, v) (or the GM deviation (a, b)),
// S = packed neighbour sums of both species.  Per species it performs the
// operations of euler_cell in the same order.
template <int MODEL>
__device__ __forceinline__ float2 euler2(float2 C, float2 S, const CoefF &c) {
    if (MODEL == RD_FHN) {
        const float u = C.x, v = C.y;
        float ru = fmaf(-u * u, u, u - v);
        return make_float2(fmaf(c.cu, fmaf(-4.f, u, S.x), fmaf(c.k1, ru, u)),
                           fmaf(c.be, v, fmaf(c.k2, u, c.cv * S.y)));
    } else if (MODEL == RD_GM) {
        const float a = C.x, b = C.y;
        float U = a + c.u0, V = b + c.v0;
        float t = fmaf(-c.k3, b, a + c.e0);
        float f = quot_fast(U * t, V);
        return make_float2(fmaf(c.cu, fmaf(-4.f, a, S.x), fmaf(c.k2, f, a)),
                           fmaf(c.be, b, fmaf(c.k2 * a, a + c.tu0, fmaf(c.cv, S.y, c.k2e1))));
    } else if (MODEL == RD_BZ) {
        float un, vn;
        euler_cell<RD_BZ>(C.x, C.y, S.x, S.y, c, un, vn);
        return make_float2(un, vn);
    } else {
        const float2 L = __ffma2_rn(make_float2(-4.f, -4.f), C, S);
        return __ffma2_rn(make_float2(c.cu, c.cv), L, C);
    }
}

template <int G, int TY, int TX>
__device__ __forceinline__ void halo2_put(float2 *hb, int tx, int ty, const float2 (&w)[TY][TX]) {
    constexpr int NY = Tiling2<G, TY, TX>::NY;
    st_row2<TX>(hb + (0 * NY + ty) * G + tx * TX, w[0]);
    st_row2<TX>(hb + (1 * NY + ty) * G + tx * TX, w[TY - 1]);
}

// One explicit Euler step of a packed tile (after halo2_put and a barrier).
template <int MODEL, int G, int TY, int TX>
__device__ __forceinline__ void tile2_step(const float2 *hb, int tx, int ty, float2 (&w)[TY][TX], const CoefF &cf) {
    constexpr int NX = Tiling2<G, TY, TX>::NX, NY = Tiling2<G, TY, TX>::NY;
    float2 pw[TX];
    if (ty > 0) {
        ld_row2<TX>(hb + (1 * NY + ty - 1) * G + tx * TX, pw);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) pw[c] = w[0][c];
    }
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        float2 sw[TX];
        if (i + 1 < TY) {
#pragma unroll
            for (int c = 0; c < TX; ++c) sw[c] = w[i + 1][c];
        } else if (ty < NY - 1) {
            ld_row2<TX>(hb + (0 * NY + ty + 1) * G + tx * TX, sw);
        } else {
#pragma unroll
            for (int c = 0; c < TX; ++c) sw[c] = w[TY - 1][c];
        }
        float2 west, east;
        west.x = __shfl_up_sync(0xffffffffu, w[i][TX - 1].x, 1, NX);
        west.y = __shfl_up_sync(0xffffffffu, w[i][TX - 1].y, 1, NX);
        east.x = __shfl_down_sync(0xffffffffu, w[i][0].x, 1, NX);
        east.y = __shfl_down_sync(0xffffffffu, w[i][0].y, 1, NX);
        if (tx == 0) west = w[i][0];
        if (tx == NX - 1) east = w[i][TX - 1];
        float2 cw[TX];
#pragma unroll
        for (int c = 0; c < TX; ++c) cw[c] = w[i][c];
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            float2 Wn = c > 0 ? cw[c - 1] : west;
            float2 En = c < TX - 1 ? cw[c + 1] : east;
            float2 S = __fadd2_rn(__fadd2_rn(pw[c], sw[c]), __fadd2_rn(Wn, En));
            w[i][c] = euler2<MODEL>(cw[c], S, cf);
        }
#pragma unroll
        for (int c = 0; c < TX; ++c) pw[c] = cw[c];
    }
}


// ---------------------------------------------------------------------------
// Packed rotating serpentine tiles: the rotating tiles above with each node's
// (u, v) in one float2, so the neighbour sums of both species are three
// paired adds (add.f32x2) instead of six, and the reaction update is euler2
// (the operations of euler_cell in the same order).  Per node the
// arithmetic is that of tile_step_rot, so the fields are bit-identical.
// Halo ring: [buf 2][edge 2][NY][G] float2 in register order; within a
// tile row, chunk h (nodes 2h, 2h+1 of every lane) of lane tx sits at float4
// index h NX + tx, so each 16-byte store or load of a warp covers one
// contiguous 512-byte run.
// ---------------------------------------------------------------------------
template <int NX, int TX>
__device__ __forceinline__ void st_row2s(float2 *row, int tx, const float2 (&a)[TX]) {
#pragma unroll
    for (int h = 0; h < TX / 2; ++h)
        *reinterpret_cast<float4 *>(row + 2 * (h * NX + tx)) =
            make_float4(a[2 * h].x, a[2 * h].y, a[2 * h + 1].x, a[2 * h + 1].y);
}

template <int NX, int TX>
__device__ __forceinline__ void ld_row2s(const float2 *row, int tx, float2 (&a)[TX]) {
#pragma unroll
    for (int h = 0; h < TX / 2; ++h) {
        const float4 t = *reinterpret_cast<const float4 *>(row + 2 * (h * NX + tx));
        a[2 * h] = make_float2(t.x, t.y);
        a[2 * h + 1] = make_float2(t.z, t.w);
    }
}

template <int G, int TY, int TX, int OFF>
__device__ __forceinline__ void halo2_put_rot(float2 *hb, int tx, int ty, const float2 (&w)[TY + 1][TX]) {
    constexpr int NY = Tiling2<G, TY, TX>::NY, NX = Tiling2<G, TY, TX>::NX, R = TY + 1;
    st_row2s<NX, TX>(hb + (0 * NY + ty) * G, tx, w[OFF % R]);
    st_row2s<NX, TX>(hb + (1 * NY + ty) * G, tx, w[(TY - 1 + OFF) % R]);
}

template <int MODEL, int G, int TY, int TX, int OFF>
__device__ __forceinline__ void tile2_step_rot(const float2 *hb, int tx, int ty, int src, float2 (&w)[TY + 1][TX],
                                               const CoefF &cf) {
    constexpr int NY = Tiling2<G, TY, TX>::NY, NX = Tiling2<G, TY, TX>::NX, R = TY + 1;
    float2 n0[TX];   // north neighbours of row 0: halo, or the row itself at the top edge
    if (ty > 0) {
        ld_row2s<NX, TX>(hb + (1 * NY + ty - 1) * G, tx, n0);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) n0[c] = w[OFF % R][c];
    }
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        const int pr = (i + OFF) % R;            // old row i
        const int qr = (i + OFF + R - 1) % R;    // old row i - 1 (free slot for i = 0): receives new row i
        const int sr = (i + 1 + OFF) % R;        // old row i + 1
        float2 sl[TX];                           // south neighbours of the last row
        if (i == TY - 1) {
            if (ty < NY - 1) {
                ld_row2s<NX, TX>(hb + (0 * NY + ty + 1) * G, tx, sl);
            } else {
#pragma unroll
                for (int c = 0; c < TX; ++c) sl[c] = w[pr][c];
            }
        }
        float2 x0, x1;
        x0.x = __shfl_xor_sync(0xffffffffu, w[pr][0].x, 1);
        x0.y = __shfl_xor_sync(0xffffffffu, w[pr][0].y, 1);
        x1.x = __shfl_sync(0xffffffffu, w[pr][TX - 1].x, src);
        x1.y = __shfl_sync(0xffffffffu, w[pr][TX - 1].y, src);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            const float2 N = i == 0 ? n0[c] : w[qr][c];
            const float2 S = i == TY - 1 ? sl[c] : w[sr][c];
            const float2 L = c > 0 ? w[pr][c - 1] : x0, E = c < TX - 1 ? w[pr][c + 1] : x1;
            const float2 sum = __fadd2_rn(__fadd2_rn(N, S), __fadd2_rn(L, E));
            w[qr][c] = euler2<MODEL>(w[pr][c], sum, cf);
        }
    }
}

}  // namespace rdcil
