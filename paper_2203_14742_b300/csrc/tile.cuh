// Register-tile helpers shared by the resident forward stepper and the
// resident adjoint stepper.
//
// A G x G field is split into TY x TX tiles, one per thread: NX = G/TX
// threads along x (a power of two <= 32, so a warp holds whole tile rows and
// the east/west neighbours of a tile edge are shuffle lanes), NY = G/TY
// along y.  North/south tile edges go through a double-buffered shared
// memory ring halo[buf 2][species 2][edge 2][NY][G] (one barrier per step).
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
    if constexpr (TX == 4) {
        *reinterpret_cast<float4 *>(dst) = make_float4(a[0], a[1], a[2], a[3]);
    } else if constexpr (TX == 2) {
        *reinterpret_cast<float2 *>(dst) = make_float2(a[0], a[1]);
    } else {
#pragma unroll
        for (int c = 0; c < TX; ++c) dst[c] = a[c];
    }
}

template <int TX>
__device__ __forceinline__ void ld_row(const float *src, float (&a)[TX]) {
    if constexpr (TX == 4) {
        float4 t = *reinterpret_cast<const float4 *>(src);
        a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
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
//   FHN: k2 = eps dt, k3 = a;   GM: k2 = rho dt, k3 = mu.
struct CoefF {
    float cu, cv, k1, k2, k3;
};

inline CoefF make_coef(const GroupDev &g) {
    double g1 = (double)(g.G - 1);
    double h2 = g1 * g1;
    CoefF c;
    c.cu = (float)(g.p[0] * g.dt * h2);
    c.cv = (float)(g.p[1] * g.dt * h2);
    c.k1 = (float)g.dt;
    if (g.model == RD_FHN || g.model == RD_GM) {
        c.k2 = (float)(g.p[2] * g.dt);
        c.k3 = (float)g.p[3];
    } else {
        c.k2 = 0.f;
        c.k3 = 0.f;
    }
    return c;
}

// One explicit Euler update of a node given the unscaled 5-point sums
// lu = (N + S + W + E - 4 c) for both species.
template <int MODEL>
__device__ __forceinline__ void euler_cell(float u, float v, float lu, float lv, const CoefF &c, float &un,
                                           float &vn) {
    if (MODEL == RD_FHN) {
        // u + dt (Du Lap u + u - u^3 - v),  v + dt (Dv Lap v + eps (u - a v))
        float ru = fmaf(-u * u, u, u - v);
        un = fmaf(c.cu, lu, fmaf(c.k1, ru, u));
        vn = fmaf(c.cv, lv, fmaf(c.k2, fmaf(-c.k3, v, u), v));
    } else if (MODEL == RD_GM) {
        // u + dt (Du Lap u + rho (u^2/v - mu u)),  v + dt (Dv Lap v + rho (u^2 - v))
        float uu = u * u;
        float q = __fdividef(uu, v);
        un = fmaf(c.cu, lu, fmaf(c.k2, fmaf(-c.k3, u, q), u));
        vn = fmaf(c.cv, lv, fmaf(c.k2, uu - v, v));
    } else {
        un = fmaf(c.cu, lu, u);
        vn = fmaf(c.cv, lv, v);
    }
}

// One explicit Euler step of a whole register tile (reads halo buffer hb
// after the barrier that follows halo_put).
template <int MODEL, int G, int TY, int TX>
__device__ __forceinline__ void tile_step(const float *hb, int tx, int ty, float (&u)[TY][TX], float (&v)[TY][TX],
                                          const CoefF &cf) {
    constexpr int NX = Tiling<G, TY, TX>::NX;
    float pu[TX], pv[TX];
    halo_north<G, TY, TX>(hb, tx, ty, u, v, pu, pv);
#pragma unroll
    for (int i = 0; i < TY; ++i) {
        float su[TX], sv[TX];
        row_south<G, TY, TX>(hb, tx, ty, i, u, v, su, sv);
        float wu, eu, wv, ev;
        row_west_east<NX>(tx, u[i][0], u[i][TX - 1], wu, eu);
        row_west_east<NX>(tx, v[i][0], v[i][TX - 1], wv, ev);
        float cu_[TX], cv_[TX];
#pragma unroll
        for (int c = 0; c < TX; ++c) { cu_[c] = u[i][c]; cv_[c] = v[i][c]; }
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            float Wu = c > 0 ? cu_[c - 1] : wu, Eu = c < TX - 1 ? cu_[c + 1] : eu;
            float Wv = c > 0 ? cv_[c - 1] : wv, Ev = c < TX - 1 ? cv_[c + 1] : ev;
            float lu = fmaf(-4.f, cu_[c], (pu[c] + su[c]) + (Wu + Eu));
            float lv = fmaf(-4.f, cv_[c], (pv[c] + sv[c]) + (Wv + Ev));
            euler_cell<MODEL>(cu_[c], cv_[c], lu, lv, cf, u[i][c], v[i][c]);
        }
#pragma unroll
        for (int c = 0; c < TX; ++c) { pu[c] = cu_[c]; pv[c] = cv_[c]; }
    }
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

}  // namespace rdcil
