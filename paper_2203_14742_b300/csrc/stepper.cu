// Reaction-diffusion initial state and explicit Euler steppers.
//
// Paper (arXiv 2203.14742): kinetics Sec. 4.1 (FHN eq. introduction:0, GM
// eq. gmSystem); initial state = equilibrium + U(0, delta), Sec. 4.1; method
// of lines with the 5-point Laplacian and mirrored Neumann ghosts,
// App. B.1.1; explicit Euler, Sec. 5.1 (the paper's earlier GPU solver also
// keeps one whole simulation per thread block, on-chip, for the whole run).
//
// Kernels
//   init_fields_kernel        counter-based noise, FP64 then one rounding to FP32
//   init_batch_kernel         the same for every 2-D group of a handle in one launch
//   rd_resident_*_kernel      one realisation per CTA, the whole field held in
//                             registers as TYxTX tiles per thread for the whole
//                             run; north/south tile edges exchanged through a
//                             double-buffered shared-memory ring (one barrier
//                             per step), east/west edges through warp shuffles
//                             (serpentine column order, see tile.cuh); FP64
//                             residual reduced with warp shuffles at exit.
//                             Tile kinds: _scalar (u, v tiles), plain
//                             (packed (u, v) float2 tiles; also the adjoint's
//                             recording pass), _rot (rows in TY + 1 rotating
//                             slots), _rot2 (packed and rotating)
//   rd_batch_kernel           persistent: every group of a handle in one
//                             launch, work units longest first from a device
//                             queue (one 128^2 or two smaller realisations per
//                             512-thread CTA)
//   rd_reference_step_kernel  one cell per thread, one Euler step per launch
//                             (the plain paths for comparison)
//   rd_f64_step_kernel        FP64 in the paper's operation order, no FMA
#include <algorithm>
#include <cstdio>
#include <vector>
#include "tile.cuh"

namespace rdcil {

// ---------------------------------------------------------------------------
// initial state
// ---------------------------------------------------------------------------
// Element i of a group's initial state (i = (r*2 + s)*cells + c is exactly
// the generator counter): equilibrium + lo + (hi - lo) U, U = the top 53
// bits of SplitMix64 output i times 2^-53, in FP64, rounded once.
__device__ __forceinline__ float init_value(int64_t i, int64_t cells, uint64_t seed, double x0u, double x0v,
                                            double lo, double hi) {
    int64_t rs = i / cells;
    int s = (int)(rs & 1);
    uint64_t z = splitmix64_at(seed, (uint64_t)i);
    double U = __dmul_rn(__ull2double_rn(z >> 11), 1.1102230246251565404e-16);  // 2^-53
    double span = __dsub_rn(hi, lo);
    double t = __dmul_rn(span, U);
    double t2 = __dadd_rn(lo, t);
    double v = __dadd_rn(s ? x0v : x0u, t2);
    return __double2float_rn(v);
}

__global__ void init_fields_kernel(float *__restrict__ out, int64_t n_total, int64_t cells,
                                   uint64_t seed, double x0u, double x0v, double lo, double hi) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total; i += stride)
        out[i] = init_value(i, cells, seed, x0u, x0v, lo, hi);
}

// Several groups' initial states in one launch (blockIdx.y = item), each
// item's values taken on the host at launch time exactly as for the
// single-group launch, passed by value.
struct InitItem {
    int64_t offset, n, cells;
    uint64_t seed;
    double u0, v0, lo, hi;
};
constexpr int INIT_MAX = 120;
struct InitBatch {
    InitItem item[INIT_MAX];
};
static_assert(sizeof(InitBatch) <= 8192, "kernel parameter table");

__global__ void init_batch_kernel(float *__restrict__ fields, const __grid_constant__ InitBatch b) {
    const InitItem &it = b.item[blockIdx.y];
    float *out = fields + it.offset;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < it.n; i += stride)
        out[i] = init_value(i, it.cells, it.seed, it.u0, it.v0, it.lo, it.hi);
}

static void equilibrium(const GroupDev &g, double &u0, double &v0) {
    if (g.model == RD_GM) {
        volatile double a = 1.0 / g.p[3];
        u0 = a;
        v0 = a * a;
    } else if (g.model == RD_BZ) {
        volatile double q = g.p[3] / g.p[2];
        u0 = g.p[2];
        v0 = q;
    } else {
        u0 = 0.0;
        v0 = 0.0;
    }
}

// every group of a handle: the 2-D groups INIT_MAX at a time in one launch,
// each RD-ODE group in its own
rd_status launch_init_all(const GroupDev *groups, int n_groups, float *fields, cudaStream_t s) {
    InitBatch b;
    int cnt = 0;
    int64_t most = 0;
    auto flush = [&]() -> rd_status {
        if (cnt == 0) return RD_OK;
        const int block = 256;
        int64_t gx = (most + block - 1) / block;
        if (gx > 148 * 4) gx = 148 * 4;
        init_batch_kernel<<<dim3((unsigned)gx, (unsigned)cnt), block, 0, s>>>(fields, b);
        note_launch();
        cnt = 0;
        most = 0;
        return cuda_status(cudaGetLastError());
    };
    for (int i = 0; i < n_groups; ++i) {
        const GroupDev &g = groups[i];
        if (g.model == RD_RDODE) {
            rd_status st = launch_rdode_init(g, fields, s);
            if (st) return st;
            continue;
        }
        double u0, v0;
        equilibrium(g, u0, v0);
        InitItem &it = b.item[cnt++];
        it.offset = g.field_offset;
        it.cells = (int64_t)g.G * g.G;
        it.n = (int64_t)g.n_real * 2 * it.cells;
        it.seed = g.seed;
        it.u0 = u0;
        it.v0 = v0;
        it.lo = g.noise_lo;
        it.hi = g.noise_hi;
        most = std::max(most, it.n);
        if (cnt == INIT_MAX) {
            rd_status st = flush();
            if (st) return st;
        }
    }
    return flush();
}

rd_status launch_init_fields(const GroupDev &g, float *fields, cudaStream_t s) {
    if (g.model == RD_RDODE) return launch_rdode_init(g, fields, s);
    double u0, v0;
    equilibrium(g, u0, v0);
    int64_t cells = (int64_t)g.G * g.G;
    int64_t n = (int64_t)g.n_real * 2 * cells;
    int block = 256;
    int64_t grid = (n + block - 1) / block;
    if (grid > 148 * 32) grid = 148 * 32;
    init_fields_kernel<<<(unsigned)grid, block, 0, s>>>(fields + g.field_offset, n, cells, g.seed,
                                                        u0, v0, g.noise_lo, g.noise_hi);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Resident stepper: one realisation per CTA, the field held in registers as
// packed (u, v) tiles for the whole run.  RECORD = true stores the state
// before every step into traj[n] (n = 0..steps-1, each 2*G*G floats per
// realisation, realisation stride traj_stride) for the adjoint's segment
// recomputation.
// ---------------------------------------------------------------------------
template <int MODEL, int G, int TY, int TX, bool RECORD>
__global__ void __launch_bounds__(Tiling2<G, TY, TX>::NT, 1)
rd_resident_kernel(float *__restrict__ fields, int64_t field_offset, int64_t steps, CoefF cf,
                   double p0, double p1, double p2, double p3, double *__restrict__ residual,
                   uint32_t *__restrict__ status, float *__restrict__ traj, int64_t traj_stride) {
    using T = Tiling2<G, TY, TX>;
    constexpr int NX = T::NX, NY = T::NY;
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);

    const int tid = threadIdx.x;
    const int tx = tid % NX, ty = tid / NX;
    const int r = blockIdx.x;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;

    float2 w[TY][TX];
    tile2_load<G, TY, TX>(base, tx, ty, w);
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) w[i][c] = to_state2<MODEL>(w[i][c], cf);

    for (int64_t n = 0; n < steps; ++n) {
        if (RECORD) {
            // state before this step, as stored fields, one tile row at a time
            float *dst = traj + (int64_t)r * traj_stride + n * 2 * G * G;
#pragma unroll
            for (int i = 0; i < TY; ++i) {
                float2 f[TX];
#pragma unroll
                for (int c = 0; c < TX; ++c) f[c] = from_state2<MODEL>(w[i][c], cf);
                st_row_g<G, TX>(dst, ty * TY + i, tx * TX, f);
            }
        }
        float2 *hb = sm + (int)(n & 1) * (T::HALO_F2 / 2);
        halo2_put<G, TY, TX>(hb, tx, ty, w);
        __syncthreads();
        tile2_step<MODEL, G, TY, TX>(hb, tx, ty, w, cf);
    }
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) w[i][c] = from_state2<MODEL>(w[i][c], cf);
    tile2_store<G, TY, TX>(base, tx, ty, w);
    if (RECORD) return;

    // ---- FP64 steady-state residual of the final (stored FP32) state -----
    residual_from_global<MODEL, G>(base, p0, p1, p2, p3, residual, status, r, sm);
}

// ---------------------------------------------------------------------------
// The same stepper with separate u and v register tiles (scalar FP32 issue).
// Per node it performs exactly the packed kernel's operations, lane by lane,
// so its fields are bit-identical; it trades issue slots for shorter
// dependency latency (packed f32x2 instructions occupy the FMA pipe for two
// cycles on this GPU).
// ---------------------------------------------------------------------------
// One realisation r of a group, by a whole CTA of Tiling<G,TY,TX>::NT
// threads; sm = the halo ring (Tiling::SMEM bytes).
// sy: the threads that run this realisation (the whole CTA, or one half of
// a 512-thread CTA in the persistent launch), Tiling::NT of them.
template <int MODEL, int G, int TY, int TX, class Sync = SyncAll>
__device__ __forceinline__ void run_scalar(float *__restrict__ fields, int64_t field_offset, int r, int64_t steps,
                                           const CoefF &cf, double p0, double p1, double p2, double p3,
                                           double *__restrict__ residual, uint32_t *__restrict__ status,
                                           float *sm, Sync sy = Sync{}) {
    using T = Tiling<G, TY, TX>;
    constexpr int NX = T::NX;
    const int tid = sy.tid();
    const int tx = tid % NX, ty = tid / NX;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;
    float u[TY][TX], v[TY][TX];
    tile_load_s<G, TY, TX>(base, tx, ty, u, v);
    tile_to_state<MODEL, TY, TX>(u, v, cf);
    const int src = serp_src<NX>(tx);
    for (int64_t n = 0; n < steps; ++n) {
        float *hb = sm + (int)(n & 1) * (T::HALO_FLOATS / 2);
        halo_put<G, TY, TX>(hb, tx, ty, u, v);
        sy.sync();
        tile_step_s<MODEL, G, TY, TX>(hb, tx, ty, src, u, v, cf);
    }
    tile_from_state<MODEL, TY, TX>(u, v, cf);
    tile_store_s<G, TY, TX>(base, tx, ty, u, v);
    residual_from_global<MODEL, G, Sync>(base, p0, p1, p2, p3, residual, status, r, sm, sy);
}

// The same with rotating tiles (tile.cuh): R = TY + 1 steps unrolled with
// the slot offsets 0, R-1, ..., 1; a step count that is not a multiple of R
// leaves the loop after the step that reaches it, and the final offset
// selects how the rows are stored.
template <int MODEL, int G, int TY, int TX, int OFF, class Sync>
__device__ __forceinline__ void rot_one(float *sm, int64_t n, int tx, int ty, int src, float (&u)[TY + 1][TX],
                                        float (&v)[TY + 1][TX], const CoefF &cf, Sync sy) {
    using T = Tiling<G, TY, TX>;
    float *hb = sm + (int)(n & 1) * (T::HALO_FLOATS / 2);
    halo_put_rot<G, TY, TX, OFF>(hb, tx, ty, u, v);
    sy.sync();
    tile_step_rot<MODEL, G, TY, TX, OFF>(hb, tx, ty, src, u, v, cf);
}

// steps with offsets OFF, OFF-1, ..., 1 (then the caller's loop restarts at
// 0); returns the offset of the next step, or -1 if all were taken
template <int MODEL, int G, int TY, int TX, int OFF, class Sync>
__device__ __forceinline__ int rot_chain(float *sm, int64_t &n, int64_t steps, int tx, int ty, int src,
                                         float (&u)[TY + 1][TX], float (&v)[TY + 1][TX], const CoefF &cf,
                                         Sync sy) {
    if constexpr (OFF == 0) {
        return -1;
    } else {
        if (n >= steps) return OFF;
        rot_one<MODEL, G, TY, TX, OFF>(sm, n, tx, ty, src, u, v, cf, sy);
        ++n;
        return rot_chain<MODEL, G, TY, TX, OFF - 1>(sm, n, steps, tx, ty, src, u, v, cf, sy);
    }
}

template <int G, int TY, int TX, int OFF>
__device__ __forceinline__ void rot_store(float *base, int tx, int ty, const float (&u)[TY + 1][TX],
                                          const float (&v)[TY + 1][TX]) {
    float a[TY][TX], b[TY][TX];
#pragma unroll
    for (int i = 0; i < TY; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) {
            a[i][c] = u[(i + OFF) % (TY + 1)][c];
            b[i][c] = v[(i + OFF) % (TY + 1)][c];
        }
    tile_store_s<G, TY, TX>(base, tx, ty, a, b);
}

template <int G, int TY, int TX, int OFF>
__device__ __forceinline__ void rot_store_any(float *base, int tx, int ty, int off, const float (&u)[TY + 1][TX],
                                              const float (&v)[TY + 1][TX]) {
    if constexpr (OFF > TY) {
        return;
    } else {
        if (off == OFF) rot_store<G, TY, TX, OFF>(base, tx, ty, u, v);
        else rot_store_any<G, TY, TX, OFF + 1>(base, tx, ty, off, u, v);
    }
}

template <int MODEL, int G, int TY, int TX, class Sync = SyncAll>
__device__ __forceinline__ void run_rot(float *__restrict__ fields, int64_t field_offset, int r, int64_t steps,
                                        const CoefF &cf, double p0, double p1, double p2, double p3,
                                        double *__restrict__ residual, uint32_t *__restrict__ status, float *sm,
                                        Sync sy = Sync{}) {
    using T = Tiling<G, TY, TX>;
    constexpr int NX = T::NX, R = TY + 1;
    const int tid = sy.tid();
    const int tx = tid % NX, ty = tid / NX;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;
    float u[R][TX], v[R][TX];
    {
        float a[TY][TX], b[TY][TX];
        tile_load_s<G, TY, TX>(base, tx, ty, a, b);
        tile_to_state<MODEL, TY, TX>(a, b, cf);
#pragma unroll
        for (int i = 0; i < TY; ++i)
#pragma unroll
            for (int c = 0; c < TX; ++c) { u[i][c] = a[i][c]; v[i][c] = b[i][c]; }
#pragma unroll
        for (int c = 0; c < TX; ++c) { u[TY][c] = 0.f; v[TY][c] = 0.f; }
    }
    const int src = serp_src<NX>(tx);
    int64_t n = 0;
    int off = 0;
    for (;;) {
        if (n >= steps) { off = 0; break; }
        rot_one<MODEL, G, TY, TX, 0>(sm, n, tx, ty, src, u, v, cf, sy);
        ++n;
        const int o = rot_chain<MODEL, G, TY, TX, R - 1>(sm, n, steps, tx, ty, src, u, v, cf, sy);
        if (o >= 0) { off = o; break; }
    }
    // back from the state form, row by row in the final mapping
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) from_state<MODEL>(u[i][c], v[i][c], cf);
    rot_store_any<G, TY, TX, 0>(base, tx, ty, off, u, v);
    residual_from_global<MODEL, G, Sync>(base, p0, p1, p2, p3, residual, status, r, sm, sy);
}

// The packed form of run_rot (tile2_step_rot: (u, v) pairs, paired
// neighbour sums), bit-identical to it.
template <int MODEL, int G, int TY, int TX, int OFF, class Sync>
__device__ __forceinline__ void rot2_one(float *sm, int64_t n, int tx, int ty, int src, float2 (&w)[TY + 1][TX],
                                         const CoefF &cf, Sync sy) {
    using T = Tiling2<G, TY, TX>;
    float2 *hb = reinterpret_cast<float2 *>(sm) + (int)(n & 1) * (T::HALO_F2 / 2);
    halo2_put_rot<G, TY, TX, OFF>(hb, tx, ty, w);
    sy.sync();
    tile2_step_rot<MODEL, G, TY, TX, OFF>(hb, tx, ty, src, w, cf);
}

template <int MODEL, int G, int TY, int TX, int OFF, class Sync>
__device__ __forceinline__ int rot2_chain(float *sm, int64_t &n, int64_t steps, int tx, int ty, int src,
                                          float2 (&w)[TY + 1][TX], const CoefF &cf, Sync sy) {
    if constexpr (OFF == 0) {
        return -1;
    } else {
        if (n >= steps) return OFF;
        rot2_one<MODEL, G, TY, TX, OFF>(sm, n, tx, ty, src, w, cf, sy);
        ++n;
        return rot2_chain<MODEL, G, TY, TX, OFF - 1>(sm, n, steps, tx, ty, src, w, cf, sy);
    }
}

template <int G, int TY, int TX, int OFF>
__device__ __forceinline__ void rot2_store_any(float *base, int tx, int ty, int off, const float2 (&w)[TY + 1][TX]) {
    if constexpr (OFF > TY) {
        return;
    } else {
        if (off == OFF) {
            float a[TY][TX], b[TY][TX];
#pragma unroll
            for (int i = 0; i < TY; ++i)
#pragma unroll
                for (int c = 0; c < TX; ++c) {
                    a[i][c] = w[(i + OFF) % (TY + 1)][c].x;
                    b[i][c] = w[(i + OFF) % (TY + 1)][c].y;
                }
            tile_store_s<G, TY, TX>(base, tx, ty, a, b);
        } else {
            rot2_store_any<G, TY, TX, OFF + 1>(base, tx, ty, off, w);
        }
    }
}

template <int MODEL, int G, int TY, int TX, class Sync = SyncAll>
__device__ __forceinline__ void run_rot2(float *__restrict__ fields, int64_t field_offset, int r, int64_t steps,
                                         const CoefF &cf, double p0, double p1, double p2, double p3,
                                         double *__restrict__ residual, uint32_t *__restrict__ status, float *sm,
                                         Sync sy = Sync{}) {
    using T = Tiling<G, TY, TX>;
    static_assert(Tiling2<G, TY, TX>::SMEM == T::SMEM, "same halo ring bytes as the scalar tiles");
    constexpr int NX = T::NX, R = TY + 1;
    const int tid = sy.tid();
    const int tx = tid % NX, ty = tid / NX;
    float *base = fields + field_offset + (int64_t)r * 2 * G * G;
    float2 w[R][TX];
    {
        float a[TY][TX], b[TY][TX];
        tile_load_s<G, TY, TX>(base, tx, ty, a, b);
        tile_to_state<MODEL, TY, TX>(a, b, cf);
#pragma unroll
        for (int i = 0; i < TY; ++i)
#pragma unroll
            for (int c = 0; c < TX; ++c) w[i][c] = make_float2(a[i][c], b[i][c]);
#pragma unroll
        for (int c = 0; c < TX; ++c) w[TY][c] = make_float2(0.f, 0.f);
    }
    const int src = serp_src<NX>(tx);
    int64_t n = 0;
    int off = 0;
    for (;;) {
        if (n >= steps) { off = 0; break; }
        rot2_one<MODEL, G, TY, TX, 0>(sm, n, tx, ty, src, w, cf, sy);
        ++n;
        const int o = rot2_chain<MODEL, G, TY, TX, R - 1>(sm, n, steps, tx, ty, src, w, cf, sy);
        if (o >= 0) { off = o; break; }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int c = 0; c < TX; ++c) from_state<MODEL>(w[i][c].x, w[i][c].y, cf);
    rot2_store_any<G, TY, TX, 0>(base, tx, ty, off, w);
    residual_from_global<MODEL, G, Sync>(base, p0, p1, p2, p3, residual, status, r, sm, sy);
}

template <int MODEL, int G, int TY, int TX>
__global__ void __launch_bounds__(Tiling<G, TY, TX>::NT, 1)
rd_resident_rot2_kernel(float *__restrict__ fields, int64_t field_offset, int64_t steps, CoefF cf, double p0,
                        double p1, double p2, double p3, double *__restrict__ residual,
                        uint32_t *__restrict__ status) {
    extern __shared__ float4 smem_f4[];
    run_rot2<MODEL, G, TY, TX>(fields, field_offset, (int)blockIdx.x, steps, cf, p0, p1, p2, p3, residual, status,
                               reinterpret_cast<float *>(smem_f4));
}

template <int MODEL, int G, int TY, int TX>
__global__ void __launch_bounds__(Tiling<G, TY, TX>::NT, 1)
rd_resident_rot_kernel(float *__restrict__ fields, int64_t field_offset, int64_t steps, CoefF cf, double p0,
                       double p1, double p2, double p3, double *__restrict__ residual, uint32_t *__restrict__ status) {
    extern __shared__ float4 smem_f4[];
    run_rot<MODEL, G, TY, TX>(fields, field_offset, (int)blockIdx.x, steps, cf, p0, p1, p2, p3, residual, status,
                              reinterpret_cast<float *>(smem_f4));
}

template <int MODEL, int G, int TY, int TX>
__global__ void __launch_bounds__(Tiling<G, TY, TX>::NT, 1)
rd_resident_scalar_kernel(float *__restrict__ fields, int64_t field_offset, int64_t steps, CoefF cf,
                          double p0, double p1, double p2, double p3, double *__restrict__ residual,
                          uint32_t *__restrict__ status) {
    extern __shared__ float4 smem_f4[];
    run_scalar<MODEL, G, TY, TX>(fields, field_offset, (int)blockIdx.x, steps, cf, p0, p1, p2, p3, residual, status,
                                 reinterpret_cast<float *>(smem_f4));
}

// ---------------------------------------------------------------------------
// Tile-shape variants.  Every variant performs the same per-node arithmetic
// in the same order (only the data movement differs), so all variants give
// bit-identical fields; the choice is a pure performance knob, picked by
// rd_autotune or the default table below.
// ---------------------------------------------------------------------------
struct Variant {
    int packed, TY, TX;   // packed: 0 scalar u, v tiles; 1 float2 (u, v) tiles; 2 rotating scalar tiles;
                          // 3 rotating float2 tiles
};
static constexpr int NVAR = 8;
static constexpr Variant VAR32[NVAR] = {{0, 4, 4}, {1, 4, 4}, {0, 2, 4}, {1, 2, 4},
                                        {1, 2, 8}, {0, 2, 8}, {0, 4, 8}, {0, 2, 2}};
static constexpr Variant VAR64[NVAR] = {{2, 4, 4}, {1, 4, 4}, {0, 2, 4}, {0, 4, 4},
                                        {0, 4, 8}, {0, 8, 4}, {2, 8, 4}, {0, 8, 8}};
static constexpr Variant VAR128[NVAR] = {{3, 8, 4}, {2, 8, 4}, {1, 8, 4}, {2, 4, 8},
                                         {0, 8, 4}, {0, 8, 8}, {0, 16, 4}, {1, 16, 4}};

template <int G> constexpr Variant var_of(int i) {
    return G == 32 ? VAR32[i] : (G == 64 ? VAR64[i] : VAR128[i]);
}

static int g_choice[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // [model][G index]
static inline int gidx(int G) { return G == 32 ? 0 : (G == 64 ? 1 : 2); }

template <int MODEL, int G, int VI, bool RECORD>
static rd_status launch_variant(const GroupDev &g, float *fields, int64_t steps, double *residual,
                                uint32_t *status, float *traj, int64_t traj_stride, cudaStream_t s) {
    constexpr Variant V = var_of<G>(VI);
    CoefF cf = make_coef(g);
    double *res = residual ? residual + 2 * g.real_base : nullptr;
    if constexpr (V.packed == 3 && !RECORD) {
        using T = Tiling<G, V.TY, V.TX>;
        auto kern = rd_resident_rot2_kernel<MODEL, G, V.TY, V.TX>;
        rd_status ast = smem_attr(kern, (int)T::SMEM);
        if (ast) return ast;
        kern<<<g.n_real, T::NT, T::SMEM, s>>>(fields, g.field_offset, steps, cf, g.p[0], g.p[1], g.p[2], g.p[3],
                                              res, status);
    } else if constexpr (V.packed == 2 && !RECORD) {
        using T = Tiling<G, V.TY, V.TX>;
        auto kern = rd_resident_rot_kernel<MODEL, G, V.TY, V.TX>;
        rd_status ast = smem_attr(kern, (int)T::SMEM);
        if (ast) return ast;
        kern<<<g.n_real, T::NT, T::SMEM, s>>>(fields, g.field_offset, steps, cf, g.p[0], g.p[1], g.p[2], g.p[3],
                                              res, status);
    } else if constexpr (V.packed || RECORD) {
        using T = Tiling2<G, V.TY, V.TX>;
        auto kern = rd_resident_kernel<MODEL, G, V.TY, V.TX, RECORD>;
        rd_status ast = smem_attr(kern, (int)T::SMEM);
        if (ast) return ast;
        kern<<<g.n_real, T::NT, T::SMEM, s>>>(fields, g.field_offset, steps, cf, g.p[0], g.p[1], g.p[2], g.p[3],
                                              res, status, traj, traj_stride);
    } else {
        using T = Tiling<G, V.TY, V.TX>;
        auto kern = rd_resident_scalar_kernel<MODEL, G, V.TY, V.TX>;
        rd_status ast = smem_attr(kern, (int)T::SMEM);
        if (ast) return ast;
        kern<<<g.n_real, T::NT, T::SMEM, s>>>(fields, g.field_offset, steps, cf, g.p[0], g.p[1], g.p[2], g.p[3],
                                              res, status);
    }
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL, int G, bool RECORD>
static rd_status launch_resident(const GroupDev &g, float *fields, int64_t steps, double *residual,
                                 uint32_t *status, float *traj, int64_t traj_stride, cudaStream_t s, int vi) {
    if constexpr (RECORD) {
        // the recording pass always uses the packed shape of variant 1
        return launch_variant<MODEL, G, 1, true>(g, fields, steps, residual, status, traj, traj_stride, s);
    } else {
        switch (vi) {
            case 1: return launch_variant<MODEL, G, 1, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            case 2: return launch_variant<MODEL, G, 2, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            case 3: return launch_variant<MODEL, G, 3, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            case 4: return launch_variant<MODEL, G, 4, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            case 5: return launch_variant<MODEL, G, 5, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            case 6: return launch_variant<MODEL, G, 6, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            case 7: return launch_variant<MODEL, G, 7, false>(g, fields, steps, residual, status, traj, traj_stride, s);
            default: return launch_variant<MODEL, G, 0, false>(g, fields, steps, residual, status, traj, traj_stride, s);
        }
    }
}

template <int MODEL, bool RECORD>
static rd_status dispatch_G(const GroupDev &g, float *fields, int64_t steps, double *residual, uint32_t *status,
                            float *traj, int64_t traj_stride, cudaStream_t s, int vi) {
    switch (g.G) {
        case 32: return launch_resident<MODEL, 32, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        case 64: return launch_resident<MODEL, 64, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        case 128: return launch_resident<MODEL, 128, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        default: return RD_ERR_UNSUPPORTED;
    }
}

template <bool RECORD>
static rd_status dispatch_model(const GroupDev &g, float *fields, int64_t steps, double *residual,
                                uint32_t *status, float *traj, int64_t traj_stride, cudaStream_t s, int vi) {
    switch (g.model) {
        case RD_FHN: return dispatch_G<RD_FHN, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        case RD_GM: return dispatch_G<RD_GM, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        case RD_DIFF: return dispatch_G<RD_DIFF, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        case RD_BZ: return dispatch_G<RD_BZ, RECORD>(g, fields, steps, residual, status, traj, traj_stride, s, vi);
        default: return RD_ERR_UNSUPPORTED;
    }
}

rd_status launch_integrate_group(const GroupDev &g, float *fields, int64_t steps, double *residual,
                                 uint32_t *status, cudaStream_t s) {
    return dispatch_model<false>(g, fields, steps, residual, status, nullptr, 0, s, g_choice[g.model][gidx(g.G)]);
}

rd_status launch_integrate_variant(const GroupDev &g, float *fields, int64_t steps, double *residual,
                                   uint32_t *status, cudaStream_t s, int vi) {
    if (vi < 0 || vi >= NVAR) return RD_ERR_INVALID_ARG;
    return dispatch_model<false>(g, fields, steps, residual, status, nullptr, 0, s, vi);
}

void set_variant_choice(int model, int G, int vi) { g_choice[model][gidx(G)] = vi; }
int get_variant_choice(int model, int G) { return g_choice[model][gidx(G)]; }
int n_variants() { return NVAR; }
bool variant_shape(int G, int vi, int *packed, int *TY, int *TX) {
    if (vi < 0 || vi >= NVAR || (G != 32 && G != 64 && G != 128)) return false;
    const Variant V = G == 32 ? VAR32[vi] : (G == 64 ? VAR64[vi] : VAR128[vi]);
    *packed = V.packed;
    *TY = V.TY;
    *TX = V.TX;
    return true;
}

// traj holds, per realisation, `steps` states of 2*G*G floats back to back.
rd_status launch_record_group(const GroupDev &g, float *fields, float *traj, int64_t steps, cudaStream_t s) {
    return dispatch_model<true>(g, fields, steps, nullptr, nullptr, traj, steps * 2 * (int64_t)g.G * g.G, s, 0);
}

// ---------------------------------------------------------------------------
// Persistent batched stepper: one launch for a whole mixed batch (several
// parameter groups, models and grid sizes).  Every CTA has 512 threads and
// loops: take the next work unit from a global queue (units ordered
// longest first), integrate it to the end, repeat.  A unit is one 128x128
// realisation on all 512 threads (packed rotating 8x4 tiles: +6.5 % on FHN
// and GM 128x128 over the scalar rotating tiles), or two realisations of
// 64x64 (scalar rotating 4x4 tiles; packed measured 2-3 % slower there) or
// 32x32 (2x2 tiles) side by side, one per half of the CTA (256 threads,
// named barrier 1 + half), so every SM keeps 16 warps.  The per-node arithmetic is the same as in the per-group
// kernels, so results are bit-identical to them.
// ---------------------------------------------------------------------------
struct BatchGroup {
    CoefF cf;
    double p[4];
    int64_t field_offset, n_steps, real_base;
    int32_t model, G, n_real, pad;
};
struct BatchUnit {
    int32_t group[2], real[2];   // group[1] = -1: the second half has no item (or a 128^2 unit)
};

constexpr int BATCH_THREADS = 512;
constexpr size_t BATCH_HALF_FLOATS = Tiling<64, 4, 4>::HALO_FLOATS;   // one half's halo ring
constexpr size_t BATCH_SMEM = Tiling<128, 8, 4>::SMEM;                // = both halves' rings
static_assert(Tiling<128, 8, 4>::NT == BATCH_THREADS && Tiling<64, 4, 4>::NT == BATCH_THREADS / 2 &&
                  Tiling<32, 2, 2>::NT == BATCH_THREADS / 2, "batch tile shapes");
static_assert(2 * Tiling<64, 4, 4>::SMEM <= BATCH_SMEM && Tiling<32, 2, 2>::SMEM <= Tiling<64, 4, 4>::SMEM,
              "halo rings");

template <int MODEL>
__device__ __forceinline__ void batch_full(float *fields, const BatchGroup &g, int r, int64_t steps, double *res,
                                           uint32_t *status, float *sm) {
    run_rot2<MODEL, 128, 8, 4>(fields, g.field_offset, r, steps, g.cf, g.p[0], g.p[1], g.p[2], g.p[3], res, status,
                               sm, SyncAll{});
}

template <int MODEL>
__device__ __forceinline__ void batch_half(float *fields, const BatchGroup &g, int r, int64_t steps, double *res,
                                           uint32_t *status, float *sm, SyncHalf sy) {
    if (g.G == 64)
        run_rot<MODEL, 64, 4, 4>(fields, g.field_offset, r, steps, g.cf, g.p[0], g.p[1], g.p[2], g.p[3], res,
                                 status, sm, sy);
    else
        run_scalar<MODEL, 32, 2, 2>(fields, g.field_offset, r, steps, g.cf, g.p[0], g.p[1], g.p[2], g.p[3], res,
                                    status, sm, sy);
}

__global__ void __launch_bounds__(BATCH_THREADS, 1)
rd_batch_kernel(float *__restrict__ fields, const BatchGroup *__restrict__ groups, const BatchUnit *__restrict__ units,
                int n_units, unsigned int *__restrict__ head, int64_t steps_override, double *__restrict__ residual,
                uint32_t *__restrict__ status) {
    extern __shared__ float4 smem_f4[];
    float *sm = reinterpret_cast<float *>(smem_f4);
    __shared__ int s_unit;
    for (;;) {
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_unit;
        __syncthreads();
        if (it >= n_units) break;
        const BatchUnit w = units[it];
        const BatchGroup g0 = groups[w.group[0]];
        if (g0.G == 128) {
            const int64_t steps = steps_override >= 0 ? steps_override : g0.n_steps;
            double *res = residual ? residual + 2 * g0.real_base : nullptr;
            switch (g0.model) {
                case RD_FHN: batch_full<RD_FHN>(fields, g0, w.real[0], steps, res, status, sm); break;
                case RD_GM: batch_full<RD_GM>(fields, g0, w.real[0], steps, res, status, sm); break;
                case RD_BZ: batch_full<RD_BZ>(fields, g0, w.real[0], steps, res, status, sm); break;
                default: batch_full<RD_DIFF>(fields, g0, w.real[0], steps, res, status, sm); break;
            }
        } else {
            const int h = threadIdx.x >> 8;
            const int gi = w.group[h];
            if (gi >= 0) {   // uniform over the half
                const BatchGroup g = groups[gi];
                const int64_t steps = steps_override >= 0 ? steps_override : g.n_steps;
                double *res = residual ? residual + 2 * g.real_base : nullptr;
                float *smh = sm + h * BATCH_HALF_FLOATS;
                const SyncHalf sy{h};
                switch (g.model) {
                    case RD_FHN: batch_half<RD_FHN>(fields, g, w.real[h], steps, res, status, smh, sy); break;
                    case RD_GM: batch_half<RD_GM>(fields, g, w.real[h], steps, res, status, smh, sy); break;
                    case RD_BZ: batch_half<RD_BZ>(fields, g, w.real[h], steps, res, status, smh, sy); break;
                    default: batch_half<RD_DIFF>(fields, g, w.real[h], steps, res, status, smh, sy); break;
                }
            }
        }
        __syncthreads();
    }
}

struct BatchPlan {
    BatchGroup *d_groups = nullptr;
    BatchUnit *d_units = nullptr;
    unsigned int *d_head = nullptr;
    int n_units = 0;
    int n_sm = 148;
};

static BatchGroup batch_group_of(const GroupDev &g) {
    BatchGroup b;
    b.cf = make_coef(g);
    for (int k = 0; k < 4; ++k) b.p[k] = g.p[k];
    b.field_offset = g.field_offset;
    b.n_steps = g.n_steps;
    b.real_base = g.real_base;
    b.model = g.model;
    b.G = g.G;
    b.n_real = g.n_real;
    b.pad = 0;
    return b;
}

rd_status batch_plan_create(const GroupDev *groups, int n_groups, void **out) {
    *out = nullptr;
    std::vector<BatchGroup> bg((size_t)n_groups);
    struct Item {
        int group, real;
        double cost;
    };
    std::vector<Item> items[3];   // by grid side 32, 64, 128
    for (int i = 0; i < n_groups; ++i) {
        const GroupDev &g = groups[i];
        bg[(size_t)i] = batch_group_of(g);
        // streaming groups run on their own launches; the 1-D model is not stepped here
        if (!group_is_resident(g) || g.model == RD_RDODE) continue;
        const int gi = g.G == 32 ? 0 : (g.G == 64 ? 1 : 2);
        for (int r = 0; r < g.n_real; ++r) items[gi].push_back(Item{i, r, (double)g.G * g.G * (double)g.n_steps});
    }
    // units: a 128^2 item alone, smaller items two by two (longest with
    // longest), then all units longest first
    std::vector<std::pair<double, BatchUnit>> units;
    for (int gi = 0; gi < 3; ++gi) {
        auto &v = items[gi];
        std::stable_sort(v.begin(), v.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
        const size_t step = gi == 2 ? 1 : 2;
        for (size_t k = 0; k < v.size(); k += step) {
            BatchUnit u{{v[k].group, -1}, {v[k].real, 0}};
            if (step == 2 && k + 1 < v.size()) {
                u.group[1] = v[k + 1].group;
                u.real[1] = v[k + 1].real;
            }
            units.push_back({v[k].cost, u});
        }
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const std::pair<double, BatchUnit> &a, const std::pair<double, BatchUnit> &b) {
                         return a.first > b.first;
                     });
    std::vector<BatchUnit> uv;
    for (auto &u : units) uv.push_back(u.second);
    BatchPlan *p = new BatchPlan();
    p->n_units = (int)uv.size();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev);
    bool ok = cudaMalloc(&p->d_groups, sizeof(BatchGroup) * bg.size()) == cudaSuccess &&
              cudaMalloc(&p->d_units, sizeof(BatchUnit) * (uv.empty() ? 1 : uv.size())) == cudaSuccess &&
              cudaMalloc(&p->d_head, sizeof(unsigned int)) == cudaSuccess &&
              cudaMemcpy(p->d_groups, bg.data(), sizeof(BatchGroup) * bg.size(), cudaMemcpyHostToDevice) ==
                  cudaSuccess &&
              (uv.empty() || cudaMemcpy(p->d_units, uv.data(), sizeof(BatchUnit) * uv.size(),
                                        cudaMemcpyHostToDevice) == cudaSuccess);
    *out = p;
    return ok ? RD_OK : RD_ERR_OOM;
}

// new parameters of group i (rd_set_params); the staged copy of the
// pageable source completes before the call returns
rd_status batch_plan_set_group(void *pp, int i, const GroupDev &g, cudaStream_t s) {
    BatchPlan *p = (BatchPlan *)pp;
    if (!p) return RD_OK;
    const BatchGroup b = batch_group_of(g);
    return cuda_status(cudaMemcpyAsync(p->d_groups + i, &b, sizeof(BatchGroup), cudaMemcpyHostToDevice, s));
}

void batch_plan_free(void *pp) {
    BatchPlan *p = (BatchPlan *)pp;
    if (!p) return;
    cudaFree(p->d_groups);
    cudaFree(p->d_units);
    cudaFree(p->d_head);
    delete p;
}

rd_status launch_batch(void *pp, float *fields, int64_t steps_override, double *residual, uint32_t *status,
                       cudaStream_t s) {
    BatchPlan *p = (BatchPlan *)pp;
    if (!p) return RD_ERR_INVALID_ARG;
    if (p->n_units == 0) return RD_OK;
    {
        rd_status ast = smem_attr(rd_batch_kernel, (int)BATCH_SMEM);
        if (ast) return ast;
    }
    RD_CUDA_TRY(cudaMemsetAsync(p->d_head, 0, sizeof(unsigned int), s));
    int grid = p->n_sm < p->n_units ? p->n_sm : p->n_units;
    rd_batch_kernel<<<grid, BATCH_THREADS, BATCH_SMEM, s>>>(fields, p->d_groups, p->d_units, p->n_units, p->d_head,
                                                           steps_override, residual, status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Plain paths: one cell per thread, one Euler step per launch, reading src
// and writing dst in global memory (blockIdx.z = realisation; the
// single-realisation path launches one realisation at a time).  GM and BZ
// nodes are converted to the deviation form that euler_cell takes (the
// Laplacian of a deviation is that of the field) and back.
// ---------------------------------------------------------------------------
template <int MODEL>
__global__ void rd_reference_step_kernel(const float *__restrict__ src, float *__restrict__ dst, int G,
                                         int64_t stride, CoefF cf) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= G || y >= G) return;
    src += (int64_t)blockIdx.z * stride;
    dst += (int64_t)blockIdx.z * stride;
    const float *u = src, *v = src + G * G;
    int k = y * G + x;
    int kn = (y > 0 ? y - 1 : y) * G + x, ks = (y < G - 1 ? y + 1 : y) * G + x;
    int kw = y * G + (x > 0 ? x - 1 : x), ke = y * G + (x < G - 1 ? x + 1 : x);
    float uc = u[k], vc = v[k], un_ = u[kn], us = u[ks], uw = u[kw], ue = u[ke];
    float vn_ = v[kn], vs = v[ks], vw = v[kw], ve = v[ke];
    to_state<MODEL>(uc, vc, cf);
    to_state<MODEL>(un_, vn_, cf);
    to_state<MODEL>(us, vs, cf);
    to_state<MODEL>(uw, vw, cf);
    to_state<MODEL>(ue, ve, cf);
    float nu = (un_ + us) + (uw + ue);
    float nv = (vn_ + vs) + (vw + ve);
    float un, vn;
    euler_cell<MODEL>(uc, vc, nu, nv, cf, un, vn);
    from_state<MODEL>(un, vn, cf);
    dst[k] = un;
    dst[G * G + k] = vn;
}

// n_at_once realisations per launch (1: the single-realisation path; n_real:
// the whole group); tmp holds 2 G^2 n_at_once floats
static rd_status plain_steps(const GroupDev &g, float *fields, float *tmp, int64_t steps, int n_at_once,
                             cudaStream_t s) {
    CoefF cf = make_coef(g);
    const int64_t m = 2 * (int64_t)g.G * g.G;
    for (int r0 = 0; r0 < g.n_real; r0 += n_at_once) {
        const int nr = min(n_at_once, g.n_real - r0);
        dim3 blk(32, 8), grd((g.G + 31) / 32, (g.G + 7) / 8, nr);
        float *a = fields + g.field_offset + r0 * m;
        for (int64_t n = 0; n < steps; ++n) {
            const float *src = (n & 1) ? tmp : a;
            float *dst = (n & 1) ? a : tmp;
            switch (g.model) {
                case RD_FHN: rd_reference_step_kernel<RD_FHN><<<grd, blk, 0, s>>>(src, dst, g.G, m, cf); break;
                case RD_GM: rd_reference_step_kernel<RD_GM><<<grd, blk, 0, s>>>(src, dst, g.G, m, cf); break;
                case RD_BZ: rd_reference_step_kernel<RD_BZ><<<grd, blk, 0, s>>>(src, dst, g.G, m, cf); break;
                default: rd_reference_step_kernel<RD_DIFF><<<grd, blk, 0, s>>>(src, dst, g.G, m, cf); break;
            }
            note_launch();
        }
        if (steps & 1) RD_CUDA_TRY(cudaMemcpyAsync(a, tmp, nr * m * sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
    return cuda_status(cudaGetLastError());
}

rd_status launch_integrate_reference(const GroupDev &g, float *fields, float *tmp, int64_t steps,
                                     cudaStream_t s) {
    return plain_steps(g, fields, tmp, steps, 1, s);
}

rd_status launch_integrate_plain(const GroupDev &g, float *fields, float *tmp, int64_t steps, cudaStream_t s) {
    if (g.n_real > 65535) return RD_ERR_UNSUPPORTED;
    return plain_steps(g, fields, tmp, steps, g.n_real, s);
}

// ---------------------------------------------------------------------------
// FP64 path in the plain operation order (no fused multiply-add):
//   lap = ((((w_{x+1} + w_{x-1}) + w_{y+1}) + w_{y-1}) - 4 w) * (G-1)^2
//   F_u = Du*lap_u + R_u,  w <- w + dt*F
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lap64(const double *w, int G, int y, int x) {
    double c = w[y * G + x];
    double xp = (x + 1 < G) ? w[y * G + x + 1] : c;
    double xm = (x - 1 >= 0) ? w[y * G + x - 1] : c;
    double yp = (y + 1 < G) ? w[(y + 1) * G + x] : c;
    double ym = (y - 1 >= 0) ? w[(y - 1) * G + x] : c;
    double g1 = (double)(G - 1);
    double sum = __dadd_rn(__dadd_rn(__dadd_rn(xp, xm), yp), ym);
    return __dmul_rn(__dsub_rn(sum, __dmul_rn(4.0, c)), __dmul_rn(g1, g1));
}

__global__ void rd_f64_step_kernel(const double *__restrict__ src, double *__restrict__ dst, int G,
                                   int n_real, int model, double dt, double p0, double p1, double p2,
                                   double p3) {
    int64_t cells = (int64_t)G * G;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cells * n_real) return;
    int64_t r = i / cells;
    int k = (int)(i - r * cells);
    int y = k / G, x = k - y * G;
    const double *u = src + r * 2 * cells, *v = u + cells;
    double lu = lap64(u, G, y, x), lv = lap64(v, G, y, x);
    double du = __dmul_rn(p0, lu), dv = __dmul_rn(p1, lv);
    double uk = u[k], vk = v[k], ru, rv;
    if (model == RD_FHN) {
        double u3 = __dmul_rn(__dmul_rn(uk, uk), uk);
        ru = __dsub_rn(__dsub_rn(uk, u3), vk);
        rv = __dmul_rn(p2, __dsub_rn(uk, __dmul_rn(p3, vk)));
    } else if (model == RD_GM) {
        double uu = __dmul_rn(uk, uk);
        double q = __ddiv_rn(uu, vk);
        ru = __dmul_rn(p2, __dsub_rn(q, __dmul_rn(p3, uk)));
        rv = __dmul_rn(p2, __dsub_rn(uu, vk));
    } else if (model == RD_BZ) {
        double uuv = __dmul_rn(__dmul_rn(uk, uk), vk);
        double bu = __dmul_rn(__dadd_rn(p3, 1.0), uk);
        ru = __dadd_rn(__dsub_rn(p2, bu), uuv);
        rv = __dsub_rn(__dmul_rn(p3, uk), uuv);
    } else {
        ru = 0.0;
        rv = 0.0;
    }
    double Fu = __dadd_rn(du, ru), Fv = __dadd_rn(dv, rv);
    double *ou = dst + r * 2 * cells, *ov = ou + cells;
    ou[k] = __dadd_rn(uk, __dmul_rn(dt, Fu));
    ov[k] = __dadd_rn(vk, __dmul_rn(dt, Fv));
}

rd_status launch_integrate_f64(const GroupDev &g, double *fields, double *tmp, int64_t steps,
                               cudaStream_t s) {
    int64_t m = 2 * (int64_t)g.G * g.G;
    int64_t n = (int64_t)g.G * g.G * g.n_real;
    double *a = fields + g.field_offset;
    double *b = tmp + g.field_offset;
    int block = 256;
    unsigned grid = (unsigned)((n + block - 1) / block);
    for (int64_t k = 0; k < steps; ++k) {
        const double *src = (k & 1) ? b : a;
        double *dst = (k & 1) ? a : b;
        rd_f64_step_kernel<<<grid, block, 0, s>>>(src, dst, g.G, g.n_real, g.model, g.dt, g.p[0], g.p[1],
                                                  g.p[2], g.p[3]);
        note_launch();
    }
    if (steps & 1)
        RD_CUDA_TRY(cudaMemcpyAsync(a, b, (size_t)(m * g.n_real) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return cuda_status(cudaGetLastError());
}

}  // namespace rdcil
