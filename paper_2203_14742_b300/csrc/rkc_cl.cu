// Adaptive stabilised second-order Runge-Kutta integration (App. B.2) of
// grids that one SM cannot hold (G = 128): a thread-block cluster of CL = 4
// CTAs integrates one realisation, CTA rank c owning rows c*G/4 .. (c+1)*G/4
// - 1.  The arithmetic per node is that of rd_rkc_kernel (rkc.cu): the stage
// recurrence on increments, every RHS evaluation of a step as F(Y_0) +
// dF(increment), the state held compensated.
//
// B300 design.  Each CTA keeps its rows in registers (4 x 4 nodes per
// thread, 256 threads) and its compensation in shared memory.  A stage's
// halo exchange writes the tile edges into the CTA's own ring (a split
// CTA-scope mbarrier orders them) and sends the CTA's first and last rows
// into its neighbours' shared memory with st.async, whose bytes complete a
// transaction mbarrier of the receiving CTA: only the warp that reads a
// neighbour's row waits for it, and no thread fences at cluster scope.  The
// exchange of F(Y_0) at the start of a step, which also reads the
// neighbours' compensation arrays, keeps a cluster barrier.  The step control is taken by
// CTA 0 alone: every CTA writes its partial error sum and spectral-radius
// bound into CTA 0's shared memory, CTA 0 decides and writes the control
// state into every CTA's shared memory, and a cluster barrier later every
// CTA reads the same decision, so the CTAs of a cluster always take the
// same path through the same barriers.
#include <cooperative_groups.h>
#include "common.cuh"
#include "tile.cuh"
#include "rkc.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace rdcil {

template <int G, int CL, int TY, int TX>
struct ClShape {
    static constexpr int R = G / CL;            // rows per CTA
    static constexpr int NX = G / TX;
    static constexpr int NY = R / TY;
    static constexpr int NT = NX * NY;
    static constexpr int RING = 2 * 2 * NY * G; // floats per ring buffer: [species][edge][NY][G]
    static constexpr int EXT = 2 * 2 * G;       // floats per buffer: [species][side 0 north, 1 south][G]
    static_assert(NX <= 32 && (NX & (NX - 1)) == 0, "tile row must fit a warp");
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    static_assert(R % TY == 0 && G % TX == 0, "tiling");
    // shared memory, byte offsets (16-byte aligned regions)
    static constexpr size_t OFF_RING = 0;
    static constexpr size_t OFF_EXT = OFF_RING + 2 * (size_t)RING * 4;
    static constexpr size_t OFF_RED = OFF_EXT + 2 * (size_t)EXT * 4;
    static constexpr size_t OFF_CLP = OFF_RED + 64 * 4;
    static constexpr size_t OFF_CTL = OFF_CLP + 16 * 4;
    static constexpr size_t OFF_BETA = (OFF_CTL + sizeof(RkcCtl) + 15) / 16 * 16;
    static constexpr size_t OFF_C0 = (OFF_BETA + RKC_STRIDE * sizeof(double) + 15) / 16 * 16;
    static constexpr size_t OFF_MB = OFF_C0 + 2 * (size_t)R * G * 4;   // ClMbar
    static constexpr size_t SMEM = OFF_MB + 64;
    static_assert(OFF_EXT % 16 == 0 && OFF_RED % 16 == 0 && OFF_CLP % 16 == 0 && OFF_CTL % 16 == 0 &&
                      OFF_BETA % 16 == 0 && OFF_C0 % 16 == 0 && OFF_MB % 16 == 0,
                  "shared-memory regions must start on 16-byte boundaries");
    static_assert(3 * CL <= 16, "cluster partials");
};

// One exchange-and-apply of a tile quantity (yu, yv): the tile edges go into
// the CTA's ring buffer hb, the CTA's first row into the CTA above (its
// south side of eb) and its last row into the CTA below (its north side)
// through distributed shared memory; then the cluster barrier is split:
// after the arrive, the interior tile rows (whose neighbours are the
// thread's own registers and its warp's shuffles) are computed while the
// barrier completes, and after the wait the first and last tile rows,
// which read the ring and the ext region.  body(i, c, nu, nv) receives the
// four neighbours (N, S, W, E) of every node, mirror ghosts at the domain
// edge.  eb: this buffer's ext region (the same offset in every CTA).
template <int G, int CL, int TY, int TX, class Body>
__device__ __forceinline__ void cl_exchange_apply(cg::cluster_group &cluster, int cr, float *hb, float *eb, int tx,
                                                  int ty, const float (&yu)[TY][TX], const float (&yv)[TY][TX],
                                                  Body body) {
    using S = ClShape<G, CL, TY, TX>;
    constexpr int NX = S::NX, NY = S::NY;
    static_assert(TY >= 3, "interior rows");
    const int x0 = tx * TX;
    st_row<TX>(hb + ((0 * 2 + 0) * NY + ty) * G + x0, yu[0]);
    st_row<TX>(hb + ((0 * 2 + 1) * NY + ty) * G + x0, yu[TY - 1]);
    st_row<TX>(hb + ((1 * 2 + 0) * NY + ty) * G + x0, yv[0]);
    st_row<TX>(hb + ((1 * 2 + 1) * NY + ty) * G + x0, yv[TY - 1]);
    if (ty == 0 && cr > 0) {
        float *up = cluster.map_shared_rank(eb, cr - 1);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            up[(0 * 2 + 1) * G + x0 + c] = yu[0][c];
            up[(1 * 2 + 1) * G + x0 + c] = yv[0][c];
        }
    }
    if (ty == NY - 1 && cr < CL - 1) {
        float *dn = cluster.map_shared_rank(eb, cr + 1);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            dn[(0 * 2 + 0) * G + x0 + c] = yu[TY - 1][c];
            dn[(1 * 2 + 0) * G + x0 + c] = yv[TY - 1][c];
        }
    }
    cluster.barrier_arrive();
    auto row = [&](int i, const float (&pu)[TX], const float (&pv)[TX], const float (&su)[TX],
                   const float (&sv)[TX]) {
        float wu, eu, wv, ev;
        row_west_east<NX>(tx, yu[i][0], yu[i][TX - 1], wu, eu);
        row_west_east<NX>(tx, yv[i][0], yv[i][TX - 1], wv, ev);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            const float Lu = c > 0 ? yu[i][c - 1] : wu, Ru = c < TX - 1 ? yu[i][c + 1] : eu;
            const float Lv = c > 0 ? yv[i][c - 1] : wv, Rv = c < TX - 1 ? yv[i][c + 1] : ev;
            body(i, c, make_float4(pu[c], su[c], Lu, Ru), make_float4(pv[c], sv[c], Lv, Rv));
        }
    };
    // interior rows: all neighbours in registers
#pragma unroll
    for (int i = 1; i < TY - 1; ++i) row(i, yu[i - 1], yv[i - 1], yu[i + 1], yv[i + 1]);
    cluster.barrier_wait();
    // first row: north from the ring / the CTA above / the mirror ghost
    {
        float pu[TX], pv[TX];
        if (ty > 0) {
            ld_row<TX>(hb + ((0 * 2 + 1) * NY + ty - 1) * G + x0, pu);
            ld_row<TX>(hb + ((1 * 2 + 1) * NY + ty - 1) * G + x0, pv);
        } else if (cr > 0) {
            ld_row<TX>(eb + (0 * 2 + 0) * G + x0, pu);
            ld_row<TX>(eb + (1 * 2 + 0) * G + x0, pv);
        } else {
#pragma unroll
            for (int c = 0; c < TX; ++c) { pu[c] = yu[0][c]; pv[c] = yv[0][c]; }
        }
        row(0, pu, pv, yu[1], yv[1]);
    }
    // last row: south from the ring / the CTA below / the mirror ghost
    {
        float su[TX], sv[TX];
        if (ty < NY - 1) {
            ld_row<TX>(hb + ((0 * 2 + 0) * NY + ty + 1) * G + x0, su);
            ld_row<TX>(hb + ((1 * 2 + 0) * NY + ty + 1) * G + x0, sv);
        } else if (cr < CL - 1) {
            ld_row<TX>(eb + (0 * 2 + 1) * G + x0, su);
            ld_row<TX>(eb + (1 * 2 + 1) * G + x0, sv);
        } else {
#pragma unroll
            for (int c = 0; c < TX; ++c) { su[c] = yu[TY - 1][c]; sv[c] = yv[TY - 1][c]; }
        }
        row(TY - 1, yu[TY - 2], yv[TY - 2], su, sv);
    }
}

// mbarriers of the stage exchanges: ring (count = threads, one phase per
// exchange), north[b] / south[b] (count 1, armed with the expected bytes by
// the lane that waits; the neighbour's st.async bytes complete them) for
// ext buffer b
struct ClMbar {
    uint64_t ring;
    uint64_t north[2];
    uint64_t south[2];
};

__device__ __forceinline__ uint32_t cl_mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// 16 bytes into another CTA's shared memory; the bytes complete a
// transaction on that CTA's mbarrier
__device__ __forceinline__ void cl_st_async(uint32_t raddr, float a, float b, float c, float d, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     raddr),
                 "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
                 "r"(rbar)
                 : "memory");
}

__device__ __forceinline__ void cl_arrive_cta(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait with acquire at cluster scope (the bytes came from another CTA)
__device__ __forceinline__ bool cl_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// The stage exchange-and-apply with mbarriers (same data, same body order as
// cl_exchange_apply).  ex = this exchange's index among the mbarrier
// exchanges (ring parity), nb[b] = uses of ext buffer b so far (its
// north/south parity); tmo: a wait gave up (later waits are skipped, the
// step reports the timeout).
template <int G, int CL, int TY, int TX, class Body>
__device__ __forceinline__ void cl_exchange_mb(int cr, float *hb, float *eb, int b, ClMbar *mb, uint32_t ex,
                                               uint32_t nbb, bool &tmo, uint32_t spin, int tx, int ty,
                                               const float (&yu)[TY][TX], const float (&yv)[TY][TX], Body body) {
    using S = ClShape<G, CL, TY, TX>;
    constexpr int NX = S::NX, NY = S::NY;
    static_assert(TY >= 3 && TX == 4, "interior rows; one 16-byte send per species");
    static_assert(NX == 32, "a tile row is one warp");
    const int x0 = tx * TX;
    const int lane = threadIdx.x & 31;
    st_row<TX>(hb + ((0 * 2 + 0) * NY + ty) * G + x0, yu[0]);
    st_row<TX>(hb + ((0 * 2 + 1) * NY + ty) * G + x0, yu[TY - 1]);
    st_row<TX>(hb + ((1 * 2 + 0) * NY + ty) * G + x0, yv[0]);
    st_row<TX>(hb + ((1 * 2 + 1) * NY + ty) * G + x0, yv[TY - 1]);
    constexpr uint32_t XB = 2 * G * 4;   // bytes of one boundary row, both species
    if (ty == 0 && cr > 0) {
        // first row -> the south side of the CTA above
        const uint32_t rank = (uint32_t)(cr - 1);
        const uint32_t rbar = cl_mapa(smem_u32(&mb->south[b]), rank);
        cl_st_async(cl_mapa(smem_u32(eb + (0 * 2 + 1) * G + x0), rank), yu[0][0], yu[0][1], yu[0][2], yu[0][3], rbar);
        cl_st_async(cl_mapa(smem_u32(eb + (1 * 2 + 1) * G + x0), rank), yv[0][0], yv[0][1], yv[0][2], yv[0][3], rbar);
        if (lane == 0) mbar_expect_tx(&mb->north[b], XB);   // this warp receives the CTA above's row
    }
    if (ty == NY - 1 && cr < CL - 1) {
        const uint32_t rank = (uint32_t)(cr + 1);
        const uint32_t rbar = cl_mapa(smem_u32(&mb->north[b]), rank);
        cl_st_async(cl_mapa(smem_u32(eb + (0 * 2 + 0) * G + x0), rank), yu[TY - 1][0], yu[TY - 1][1], yu[TY - 1][2],
                    yu[TY - 1][3], rbar);
        cl_st_async(cl_mapa(smem_u32(eb + (1 * 2 + 0) * G + x0), rank), yv[TY - 1][0], yv[TY - 1][1], yv[TY - 1][2],
                    yv[TY - 1][3], rbar);
        if (lane == 0) mbar_expect_tx(&mb->south[b], XB);
    }
    cl_arrive_cta(&mb->ring);
    auto row = [&](int i, const float (&pu)[TX], const float (&pv)[TX], const float (&su)[TX],
                   const float (&sv)[TX]) {
        float wu, eu, wv, ev;
        row_west_east<NX>(tx, yu[i][0], yu[i][TX - 1], wu, eu);
        row_west_east<NX>(tx, yv[i][0], yv[i][TX - 1], wv, ev);
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            const float Lu = c > 0 ? yu[i][c - 1] : wu, Ru = c < TX - 1 ? yu[i][c + 1] : eu;
            const float Lv = c > 0 ? yv[i][c - 1] : wv, Rv = c < TX - 1 ? yv[i][c + 1] : ev;
            body(i, c, make_float4(pu[c], su[c], Lu, Ru), make_float4(pv[c], sv[c], Lv, Rv));
        }
    };
    // interior rows: all neighbours in registers
#pragma unroll
    for (int i = 1; i < TY - 1; ++i) row(i, yu[i - 1], yv[i - 1], yu[i + 1], yv[i + 1]);
    if (!tmo && !mbar_wait(&mb->ring, ex & 1u, spin)) tmo = true;
    // first row: north from the ring / the CTA above / the mirror ghost
    {
        float pu[TX], pv[TX];
        if (ty > 0) {
            ld_row<TX>(hb + ((0 * 2 + 1) * NY + ty - 1) * G + x0, pu);
            ld_row<TX>(hb + ((1 * 2 + 1) * NY + ty - 1) * G + x0, pv);
        } else if (cr > 0) {
            if (!tmo && !cl_wait(&mb->north[b], nbb & 1u, spin)) tmo = true;
            ld_row<TX>(eb + (0 * 2 + 0) * G + x0, pu);
            ld_row<TX>(eb + (1 * 2 + 0) * G + x0, pv);
        } else {
#pragma unroll
            for (int c = 0; c < TX; ++c) { pu[c] = yu[0][c]; pv[c] = yv[0][c]; }
        }
        row(0, pu, pv, yu[1], yv[1]);
    }
    // last row: south from the ring / the CTA below / the mirror ghost
    {
        float su[TX], sv[TX];
        if (ty < NY - 1) {
            ld_row<TX>(hb + ((0 * 2 + 0) * NY + ty + 1) * G + x0, su);
            ld_row<TX>(hb + ((1 * 2 + 0) * NY + ty + 1) * G + x0, sv);
        } else if (cr < CL - 1) {
            if (!tmo && !cl_wait(&mb->south[b], nbb & 1u, spin)) tmo = true;
            ld_row<TX>(eb + (0 * 2 + 1) * G + x0, su);
            ld_row<TX>(eb + (1 * 2 + 1) * G + x0, sv);
        } else {
#pragma unroll
            for (int c = 0; c < TX; ++c) { su[c] = yu[TY - 1][c]; sv[c] = yv[TY - 1][c]; }
        }
        row(TY - 1, yu[TY - 2], yv[TY - 2], su, sv);
    }
}

template <int MODEL, int G, int CL, int TY, int TX>
__global__ void __launch_bounds__(ClShape<G, CL, TY, TX>::NT, 1)
rd_rkc_cl_kernel(float *__restrict__ fields, int64_t field_offset, RkcK k, RkcRun run, double t_end,
                 const float4 *__restrict__ tab, const double *__restrict__ beta, int64_t *__restrict__ stats,
                 double p0, double p1, double p2, double p3, double *__restrict__ residual,
                 uint32_t *__restrict__ status) {
    using S = ClShape<G, CL, TY, TX>;
    constexpr int NX = S::NX, R = S::R;
    constexpr int M = 2 * G * G;
    cg::cluster_group cluster = cg::this_cluster();
    const int cr = (int)cluster.block_rank();
    const int r = (int)(blockIdx.x / CL);
    extern __shared__ float4 smem_f4[];
    char *sb = reinterpret_cast<char *>(smem_f4);
    float *ring = reinterpret_cast<float *>(sb + S::OFF_RING);
    float *ext = reinterpret_cast<float *>(sb + S::OFF_EXT);
    float *red = reinterpret_cast<float *>(sb + S::OFF_RED);
    float *clp = reinterpret_cast<float *>(sb + S::OFF_CLP);
    RkcCtl &c = *reinterpret_cast<RkcCtl *>(sb + S::OFF_CTL);
    double *betaS = reinterpret_cast<double *>(sb + S::OFF_BETA);
    float *c0 = reinterpret_cast<float *>(sb + S::OFF_C0);     // [species][R][G], own rows
    ClMbar *mb = reinterpret_cast<ClMbar *>(sb + S::OFF_MB);
    const int tid = threadIdx.x, tx = tid % NX, ty = tid / NX;
    if (tid == 0) {
        // visible to the other CTAs through the cluster barriers that come
        // before the first stage exchange
        mbar_init(&mb->ring, S::NT);
        for (int q = 0; q < 2; ++q) {
            mbar_init(&mb->north[q], 1);
            mbar_init(&mb->south[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    bool tmo = false;                 // a stage-exchange wait gave up
    uint32_t ex = 0, nb0 = 0, nb1 = 0;   // mbarrier exchanges so far; uses of ext buffer 0 / 1
    for (int i = tid; i < RKC_STRIDE; i += blockDim.x) betaS[i] = beta[i];
    float *base = fields + field_offset + (int64_t)r * M;
    float *mine = base + (int64_t)cr * R * G;                  // this CTA's first row
    const bool adaptive = run.s_fixed < 2;
    float ku, kv;
    react_scale<MODEL>(k, ku, kv);
    // neighbours' compensation arrays (rows across the CTA boundary)
    const float *c0_up = cr > 0 ? cluster.map_shared_rank(c0, cr - 1) : nullptr;
    const float *c0_dn = cr < CL - 1 ? cluster.map_shared_rank(c0, cr + 1) : nullptr;

    float y0u[TY][TX], y0v[TY][TX], f0u[TY][TX], f0v[TY][TX];
    float d1u[TY][TX], d1v[TY][TX], d2u[TY][TX], d2v[TY][TX];
    tile_load<G, TY, TX>(mine, tx, ty, y0u, y0v);
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
            c0[R * G + node] = 0.f;
        }
    // global row of a local row, in-domain neighbour count
    auto ncount = [&](int i, int cc) {
        const int y = cr * R + ty * TY + i, x = tx * TX + cc;
        return (float)((x > 0) + (x < G - 1) + (y > 0) + (y < G - 1));
    };
    // compensation of species sp at local row y (-1 / R: the neighbours'), column x
    auto cval = [&](int sp, int y, int x) {
        if (y < 0) return cr > 0 ? c0_up[sp * R * G + (R - 1) * G + x] : c0[sp * R * G + x];
        if (y >= R) return cr < CL - 1 ? c0_dn[sp * R * G + x] : c0[sp * R * G + (R - 1) * G + x];
        return c0[sp * R * G + y * G + x];
    };
    auto lapc = [&](int sp, int y, int x) {
        const float ce = c0[sp * R * G + y * G + x];
        const float n = cval(sp, y - 1, x), so = cval(sp, y + 1, x);
        const float w = c0[sp * R * G + y * G + (x > 0 ? x - 1 : x)];
        const float e = c0[sp * R * G + y * G + (x < G - 1 ? x + 1 : x)];
        return fmaf(-4.f, ce, (n + so) + (w + e));
    };
    // the CTA's partial sums (and whether a wait gave up) to CTA 0, a cluster
    // barrier (CTA 0 then has all)
    auto to_rank0 = [&](float ss, float mx) {
        const int anyt = __syncthreads_or(tmo ? 1 : 0);
        if (tid == 0) {
            float *dst = cluster.map_shared_rank(clp, 0);
            dst[2 * cr] = ss;
            dst[2 * cr + 1] = mx;
            dst[2 * CL + cr] = anyt ? 1.f : 0.f;
        }
        cluster.sync();
    };
    auto timed_out = [&]() {
        bool t = false;
        for (int q = 0; q < CL; ++q) t |= clp[2 * CL + q] != 0.f;
        return t;
    };

    // CTA 0's control state into every CTA, a cluster barrier
    auto broadcast = [&]() {
        if (cr == 0 && tid == 0)
            for (int q = 1; q < CL; ++q) *cluster.map_shared_rank(&c, q) = c;
        cluster.sync();
    };

    int hk = 0;
    auto hbuf = [&]() { return ring + hk * S::RING; };
    auto ebuf = [&]() { return ext + hk * S::EXT; };
    // one stage exchange through the mbarriers (buffer hk), then flip
    auto xchg = [&](const float (&yu)[TY][TX], const float (&yv)[TY][TX], auto body) {
        const int b = hk;
        cl_exchange_mb<G, CL, TY, TX>(cr, hbuf(), ebuf(), b, mb, ex, b ? nb1 : nb0, tmo, MBAR_WAIT_LIMIT, tx, ty,
                                      yu, yv, body);
        ++ex;
        if (b) ++nb1;
        else ++nb0;
        hk ^= 1;
    };
    auto eval0 = [&]() {
        cl_exchange_apply<G, CL, TY, TX>(cluster, cr, hbuf(), ebuf(), tx, ty, y0u, y0v,
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
    {
        float rmax = 0.f;
        if (adaptive) {
#pragma unroll
            for (int i = 0; i < TY; ++i)
#pragma unroll
                for (int cc = 0; cc < TX; ++cc)
                    rmax = fmaxf(rmax, gersh_cell<MODEL>(y0u[i][cc] + k.u0, y0v[i][cc] + k.v0, ncount(i, cc), k));
        }
        float dummy = 0.f;
        block_reduce2(dummy, rmax, red);
        to_rank0(0.f, rmax);
        if (cr == 0 && tid == 0) {
            float rho = 0.f;
            for (int q = 0; q < CL; ++q) rho = fmaxf(rho, clp[2 * q + 1]);
            c.t = 0.0;
            c.t_end = t_end;
            c.h = run.h0;
            c.h_prev = 0.0;
            c.err_prev = 0.f;
            c.attempts = 0;
            c.n_acc = 0;
            c.n_rej = 0;
            c.n_rhs = 1;
            c.rho = rho;
            c.s = 0;
            c.s_used = 0;
            c.have_prev = 0;
            c.after_reject = 0;
            c.accept = 0;
            c.done = 0;
            c.fail = 0;
            rkc_plan(c, run, betaS);
            if (timed_out()) { c.done = 1; c.fail = 3; }
        }
        broadcast();
    }

    while (!c.done) {
        const int s = c.s;
        const float h = c.hf;
        // the coefficient row is read from the global table (uniform,
        // L1-cached loads): a stage's interior rows run before its barrier
        // completes, so a shared-memory copy would need a barrier of its own
        const float4 *row = tab + (size_t)s * RKC_STRIDE;
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
        // one stage j: D_j over dp from dl (see rkc_stage in rkc.cu)
        auto stage = [&](const float (&dlu)[TY][TX], const float (&dlv)[TY][TX], float (&dpu)[TY][TX],
                         float (&dpv)[TY][TX], int j) {
            const float4 cj = __ldg(&row[j]);
            const float mth = cj.z * h, cfh = (cj.z + cj.w) * h;
            const float mdu = mth * k.du, mdv = mth * k.dv, mru = mth * ku, mrv = mth * kv;
            xchg(dlu, dlv, [&](int i, int cc, float4 nu, float4 nv) {
                float gu = cfh * f0u[i][cc], gv = cfh * f0v[i][cc];
                if (MODEL != RD_DIFF) {
                    float dRu, dRv;
                    rhs_dparts<MODEL>(y0u[i][cc], y0v[i][cc], dlu[i][cc], dlv[i][cc], k, dRu, dRv);
                    gu = fmaf(mru, dRu, gu);
                    gv = fmaf(mrv, dRv, gv);
                }
                dpu[i][cc] = fmaf(cj.x, dlu[i][cc], fmaf(cj.y, dpu[i][cc], fmaf(mdu, lap5(dlu[i][cc], nu), gu)));
                dpv[i][cc] = fmaf(cj.x, dlv[i][cc], fmaf(cj.y, dpv[i][cc], fmaf(mdv, lap5(dlv[i][cc], nv), gv)));
            });
        };
        for (int j = 2; j <= s; j += 2) {
            stage(d1u, d1v, d2u, d2v, j);
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
            stage(d2u, d2v, d1u, d1v, j + 1);
        }
        float acc = 0.f, rmax = 0.f;
        if (adaptive) {
            const float rtol = (float)run.rtol, atol = (float)run.atol, h04 = 0.4f * h;
            xchg(d1u, d1v, [&](int i, int cc, float4 nu, float4 nv) {
                float dRu = 0.f, dRv = 0.f;
                if (MODEL != RD_DIFF) rhs_dparts<MODEL>(y0u[i][cc], y0v[i][cc], d1u[i][cc], d1v[i][cc], k, dRu, dRv);
                const float dFu = fmaf(k.du, lap5(d1u[i][cc], nu), ku * dRu);
                const float dFv = fmaf(k.dv, lap5(d1v[i][cc], nv), kv * dRv);
                const float eu = fmaf(-0.8f, d1u[i][cc], h04 * fmaf(2.f, f0u[i][cc], dFu));
                const float ev = fmaf(-0.8f, d1v[i][cc], h04 * fmaf(2.f, f0v[i][cc], dFv));
                const float U0 = y0u[i][cc] + k.u0, V0 = y0v[i][cc] + k.v0;
                const float Us = (y0u[i][cc] + d1u[i][cc]) + k.u0, Vs = (y0v[i][cc] + d1v[i][cc]) + k.v0;
                const float qu = __fdividef(eu, fmaf(rtol, fmaxf(fabsf(U0), fabsf(Us)), atol));
                const float qv = __fdividef(ev, fmaf(rtol, fmaxf(fabsf(V0), fabsf(Vs)), atol));
                acc = fmaf(qu, qu, fmaf(qv, qv, acc));
                rmax = fmaxf(rmax, gersh_cell<MODEL>(Us, Vs, ncount(i, cc), k));
            });
        }
        block_reduce2(acc, rmax, red);
        to_rank0(acc, rmax);
        if (cr == 0 && tid == 0) {
            float ss = 0.f, rho = 0.f;
            for (int q = 0; q < CL; ++q) {
                ss += clp[2 * q];
                rho = fmaxf(rho, clp[2 * q + 1]);
            }
            c.rho_new = rho;
            rkc_decide(c, run, betaS, ss, M);
            if (timed_out()) { c.accept = 0; c.done = 1; c.fail = 3; }
        }
        broadcast();
        if (c.accept) {
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
                        const float lo = c0[R * G + node] + e;
                        y0v[i][cc] = sw + lo;
                        c0[R * G + node] = lo - (y0v[i][cc] - sw);
                    }
                }
            if (!c.done) eval0();
        }
    }
    {
        CoefF cf{};
        cf.u0 = k.u0;
        cf.v0 = k.v0;
        tile_from_state<MODEL, TY, TX>(y0u, y0v, cf);
    }
    tile_store<G, TY, TX>(mine, tx, ty, y0u, y0v);
    // every CTA's rows stored (and no CTA touches another's shared memory
    // after this barrier)
    cluster.sync();
    if (cr != 0) return;
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
        if (c.fail == 3) atomicOr(status, (unsigned)ST_TIMEOUT);
    }
    residual_from_global<MODEL, G>(base, p0, p1, p2, p3, residual, status, r, ring);
}

template <int MODEL>
static rd_status launch_cl_m(const GroupDev &g, float *fields, const RkcRun &run, const float4 *tab,
                             const double *beta, int64_t *stats, double *residual, uint32_t *status, cudaStream_t s) {
    constexpr int G = 128, CL = 4, TY = 4, TX = 4;
    using S = ClShape<G, CL, TY, TX>;
    auto kern = rd_rkc_cl_kernel<MODEL, G, CL, TY, TX>;
    RD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g.n_real * CL), 1, 1);
    cfg.blockDim = dim3(S::NT, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const double t_end = run.t_end > 0.0 ? run.t_end : g.dt * (double)g.n_steps;
    RD_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, fields, g.field_offset, make_rkc_k(g), run, t_end, tab, beta,
                                   stats ? stats + 4 * g.real_base : nullptr, g.p[0], g.p[1], g.p[2], g.p[3],
                                   residual ? residual + 2 * g.real_base : nullptr, status));
    note_launch();
    return cuda_status(cudaGetLastError());
}

rd_status launch_rkc_cluster_group(const GroupDev &g, float *fields, const RkcRun &run, const float4 *tab,
                                   const double *beta, int64_t *stats, double *residual, uint32_t *status,
                                   cudaStream_t s) {
    if (g.G != 128) return RD_ERR_UNSUPPORTED;
    switch (g.model) {
        case RD_FHN: return launch_cl_m<RD_FHN>(g, fields, run, tab, beta, stats, residual, status, s);
        case RD_GM: return launch_cl_m<RD_GM>(g, fields, run, tab, beta, stats, residual, status, s);
        case RD_DIFF: return launch_cl_m<RD_DIFF>(g, fields, run, tab, beta, stats, residual, status, s);
        case RD_BZ: return launch_cl_m<RD_BZ>(g, fields, run, tab, beta, stats, residual, status, s);
        default: return RD_ERR_INVALID_ARG;
    }
}

}  // namespace rdcil
