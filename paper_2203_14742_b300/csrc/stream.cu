// Streaming Euler stepper for grids that do not fit one CTA's registers
// (any G that is a multiple of 4 other than the resident 32, 64, 128, or
// any group flagged RD_GROUP_STREAM).  Same method as the resident stepper
// (explicit Euler, 5-point Laplacian, mirrored Neumann ghosts; App. B.1.1,
// Sec. 5.1), organised around HBM:
//   * one CTA per (32 x 64 output tile, realisation); TMA
//     (cp.async.bulk.tensor.3d) loads the tile plus a halo of S rows and
//     max(4, S) columns of both species into shared memory (the column halo
//     keeps the box start 16-byte aligned; out-of-range boxes read zeros,
//     which the update never uses: at the domain edge the mirror ghost is
//     the node itself);
//   * S Euler steps run in shared memory (temporal blocking, ping-pong
//     buffers); step j updates the tile shrunk by j on every side that is
//     not a domain edge, 4 nodes per thread per pass (float4 rows; taking
//     the west / east neighbours from the neighbouring lanes by shuffle
//     measured 15 % slower at depth 4: shuffles share the shared-memory
//     pipe);
//   * the output tile goes back with float4 stores into the other HBM buffer
//     (ping-pong between the fields and a handle-owned buffer).
// Per node the arithmetic is euler_cell's, and GM / BZ stay in deviation
// form between launches, so the fields are bit-identical to the resident
// stepper's for the same group.  HBM traffic: the tile plus halo read and
// the tile written once per S steps, about (1.3 + 1) x 8 B per S
// cell-updates.
#include "tile.cuh"
#include "tma.cuh"
#include <cudaTypedefs.h>
#include <mutex>

namespace rdcil {

constexpr int ST_TX = 64, ST_TY = 32, ST_THREADS = 256;
constexpr int ST_PARTS = 64;   // residual partial sums per realisation

template <int S>
struct StreamShape {
    static constexpr int HY = S;
    static constexpr int HX = S <= 4 ? 4 : 8;
    static constexpr int SY = ST_TY + 2 * HY;
    static constexpr int SX = ST_TX + 2 * HX;
    static constexpr int PLANE = SY * SX;                  // floats of one species plane
    static constexpr int PST = (PLANE + 31) / 32 * 32;    // plane stride (128-byte multiple)
    static constexpr size_t SMEM = 4 * (size_t)PST * sizeof(float) + 128 + 16;
    static_assert(SX % 4 == 0 && SX <= 256 && SY <= 256, "TMA box");
};

bool group_is_resident(const GroupDev &g) {
    return !(g.flags & RD_GROUP_STREAM) && (g.G == 32 || g.G == 64 || g.G == 128);
}

template <int MODEL, int S>
__global__ void __launch_bounds__(ST_THREADS) rd_stream_kernel(const __grid_constant__ CUtensorMap tm_src,
                                                               float *__restrict__ dst, int G, int nsteps, CoefF cf,
                                                               int in_dev, int out_dev, uint32_t *status) {
    using SS = StreamShape<S>;
    constexpr int HY = SS::HY, HX = SS::HX, SY = SS::SY, SX = SS::SX, PST = SS::PST;
    extern __shared__ float4 smem_f4[];
    float *sm = reinterpret_cast<float *>(((uintptr_t)smem_f4 + 127) & ~(uintptr_t)127);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 4 * PST);
    const int tid = threadIdx.x;
    const int gx0 = blockIdx.x * ST_TX, gy0 = blockIdx.y * ST_TY, r = blockIdx.z;

    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar, 2u * SX * SY * sizeof(float));
        tma_load_3d(sm, &tm_src, gx0 - HX, gy0 - HY, 2 * r + 0, bar);
        tma_load_3d(sm + PST, &tm_src, gx0 - HX, gy0 - HY, 2 * r + 1, bar);
    }
    const bool got = mbar_wait(bar, 0);
    if (!__syncthreads_and(got ? 1 : 0)) {
        // let the copy land before the block's shared memory is released
        if (tid == 0) {
            mbar_wait(bar, 0);
            atomicOr(status, (unsigned)ST_TIMEOUT);
        }
        __syncthreads();
        return;
    }
    if (!in_dev && (MODEL == RD_GM || MODEL == RD_BZ)) {
        for (int e = tid; e < SY * SX; e += ST_THREADS) {
            float u = sm[e], v = sm[PST + e];
            to_state<MODEL>(u, v, cf);
            sm[e] = u;
            sm[PST + e] = v;
        }
        __syncthreads();
    }

    // local extent of the domain inside the loaded box, and which sides are
    // domain edges (mirror ghosts, no shrinking)
    const int ydl = max(0, HY - gy0), ydh = min(SY, G - gy0 + HY);
    const int xdl = max(0, HX - gx0), xdh = min(SX, G - gx0 + HX);
    const bool top = gy0 - HY <= 0, bot = gy0 + ST_TY + HY >= G;
    const bool lft = gx0 - HX <= 0, rgt = gx0 + ST_TX + HX >= G;
    int cur = 0;
    for (int j = 1; j <= nsteps; ++j) {
        const int r0 = top ? ydl : (HY - nsteps) + j;
        const int r1 = bot ? ydh : SY - (HY - nsteps) - j;
        const int c0 = (lft ? xdl : (HX - nsteps) + j) & ~3;
        const int c1 = ((rgt ? xdh : SX - (HX - nsteps) - j) + 3) & ~3;
        const float *su = sm + cur * 2 * PST, *sv = su + PST;
        float *du = sm + (cur ^ 1) * 2 * PST, *dv = du + PST;
        const int nc4 = (c1 - c0) >> 2, nrow = r1 - r0;
        for (int e = tid; e < nrow * nc4; e += ST_THREADS) {
            const int ly = r0 + e / nc4, lx = c0 + 4 * (e % nc4);
            const int gy = gy0 - HY + ly, gx = gx0 - HX + lx;
            const int k = ly * SX + lx;
            const float4 cu = *reinterpret_cast<const float4 *>(su + k);
            const float4 cv = *reinterpret_cast<const float4 *>(sv + k);
            const float4 nu = gy == 0 ? cu : *reinterpret_cast<const float4 *>(su + k - SX);
            const float4 nv = gy == 0 ? cv : *reinterpret_cast<const float4 *>(sv + k - SX);
            const float4 pu = gy == G - 1 ? cu : *reinterpret_cast<const float4 *>(su + k + SX);
            const float4 pv = gy == G - 1 ? cv : *reinterpret_cast<const float4 *>(sv + k + SX);
            const bool wm = gx == 0 || lx == 0, em = gx + 3 == G - 1 || lx + 4 >= SX;
            const float wu = wm ? cu.x : su[k - 1], wv = wm ? cv.x : sv[k - 1];
            const float eu = em ? cu.w : su[k + 4], ev = em ? cv.w : sv[k + 4];
            const float C0[4] = {cu.x, cu.y, cu.z, cu.w}, C1[4] = {cv.x, cv.y, cv.z, cv.w};
            const float N0[4] = {nu.x, nu.y, nu.z, nu.w}, N1[4] = {nv.x, nv.y, nv.z, nv.w};
            const float P0[4] = {pu.x, pu.y, pu.z, pu.w}, P1[4] = {pv.x, pv.y, pv.z, pv.w};
            float o0[4], o1[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float Wu = c > 0 ? C0[c - 1] : wu, Eu = c < 3 ? C0[c + 1] : eu;
                const float Wv = c > 0 ? C1[c - 1] : wv, Ev = c < 3 ? C1[c + 1] : ev;
                const float sumu = (N0[c] + P0[c]) + (Wu + Eu);
                const float sumv = (N1[c] + P1[c]) + (Wv + Ev);
                euler_cell<MODEL>(C0[c], C1[c], sumu, sumv, cf, o0[c], o1[c]);
            }
            *reinterpret_cast<float4 *>(du + k) = make_float4(o0[0], o0[1], o0[2], o0[3]);
            *reinterpret_cast<float4 *>(dv + k) = make_float4(o1[0], o1[1], o1[2], o1[3]);
        }
        __syncthreads();
        cur ^= 1;
    }

    // the output tile: local rows [HY, HY + 32), columns [HX, HX + 64)
    const float *su = sm + cur * 2 * PST, *sv = su + PST;
    const int64_t plane = (int64_t)G * G;
    float *ou = dst + (int64_t)(2 * r) * plane, *ov = ou + plane;
    bool bad = false;
    for (int e = tid; e < ST_TY * (ST_TX / 4); e += ST_THREADS) {
        const int ty = e / (ST_TX / 4), tx4 = e % (ST_TX / 4);
        const int gy = gy0 + ty, gx = gx0 + 4 * tx4;
        if (gy >= G || gx >= G) continue;
        const int k = (HY + ty) * SX + HX + 4 * tx4;
        float4 a = *reinterpret_cast<const float4 *>(su + k), b = *reinterpret_cast<const float4 *>(sv + k);
        if (!out_dev && (MODEL == RD_GM || MODEL == RD_BZ)) {
            from_state<MODEL>(a.x, b.x, cf);
            from_state<MODEL>(a.y, b.y, cf);
            from_state<MODEL>(a.z, b.z, cf);
            from_state<MODEL>(a.w, b.w, cf);
        }
        *reinterpret_cast<float4 *>(ou + (int64_t)gy * G + gx) = a;
        *reinterpret_cast<float4 *>(ov + (int64_t)gy * G + gx) = b;
        bad |= !(isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w) && isfinite(b.x) &&
                 isfinite(b.y) && isfinite(b.z) && isfinite(b.w));
    }
    // the last launch of a run flags a final state that is not finite
    if (!out_dev && __syncthreads_or(bad ? 1 : 0) && tid == 0) atomicOr(status, (unsigned)ST_NONFINITE);
}

// FP64 residual of the final state when asked for (as the resident
// stepper's epilogue; the last stepping launch already flags a final state
// that is not finite):
// partial max |F| and sum F^2 per (chunk, realisation), then a fixed-order
// combination per realisation.
template <int MODEL>
__global__ void __launch_bounds__(256) stream_residual_part_kernel(const float *__restrict__ f, int G, double p0,
                                                                   double p1, double p2, double p3,
                                                                   double *__restrict__ part,
                                                                   uint32_t *__restrict__ status) {
    const int c = blockIdx.x, r = blockIdx.y;
    const int64_t cells = (int64_t)G * G;
    const int64_t per = (cells + ST_PARTS - 1) / ST_PARTS;
    const int64_t k0 = (int64_t)c * per, k1 = min(cells, k0 + per);
    const float *u = f + (int64_t)(2 * r) * cells, *v = u + cells;
    const double p[4] = {p0, p1, p2, p3};
    const double h2 = (double)(G - 1) * (double)(G - 1);
    double mx = 0.0, ss = 0.0;
    bool bad = false;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const int y = (int)(k / G), x = (int)(k - (int64_t)y * G);
        const int64_t kn = (y > 0 ? k - G : k), ks = (y < G - 1 ? k + G : k);
        const int64_t kw = (x > 0 ? k - 1 : k), ke = (x < G - 1 ? k + 1 : k);
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
    __shared__ double red[2][8];
    const int anybad = __syncthreads_or(bad ? 1 : 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = mx; red[1][warp] = ss; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0, t = 0.0;
        for (int w = 0; w < 8; ++w) { m = fmax(m, red[0][w]); t += red[1][w]; }
        if (anybad) {
            atomicOr(status, (unsigned)ST_NONFINITE);
            m = t = __longlong_as_double(0x7ff8000000000000ll);   // this chunk is not finite
        }
        part[((int64_t)r * ST_PARTS + c) * 2 + 0] = m;
        part[((int64_t)r * ST_PARTS + c) * 2 + 1] = t;
    }
}

__global__ void stream_residual_final_kernel(const double *__restrict__ part, int n_real, int G,
                                             double *__restrict__ residual) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_real) return;
    double m = 0.0, t = 0.0;
    bool bad = false;
    for (int c = 0; c < ST_PARTS; ++c) {
        const double pm = part[((int64_t)r * ST_PARTS + c) * 2 + 0];
        bad |= isnan(pm);
        m = fmax(m, pm);
        t += part[((int64_t)r * ST_PARTS + c) * 2 + 1];
    }
    // as the resident epilogue: a realisation that is not finite reports NaN
    if (bad) m = t = __longlong_as_double(0x7ff8000000000000ll);
    residual[2 * r] = m;
    residual[2 * r + 1] = sqrt(t / (double)(2 * (int64_t)G * G));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 3-D view (x, y, species plane) of one group's fields, box = the tile plus
// halo of depth S.
template <int S>
static bool stream_map(CUtensorMap *m, const float *base, int G, int64_t planes) {
    using SS = StreamShape<S>;
    auto fn = encode_tiled();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)G, (cuuint64_t)G, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)G * 4, (cuuint64_t)G * G * 4};
    cuuint32_t box[3] = {(cuuint32_t)SS::SX, (cuuint32_t)SS::SY, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODEL, int S>
static rd_status stream_launch(const float *src, float *dst, const GroupDev &g, int nst, const CoefF &cf, int in_dev,
                               int out_dev, uint32_t *status, cudaStream_t s) {
    using SS = StreamShape<S>;
    CUtensorMap tm;
    if (!stream_map<S>(&tm, src, g.G, 2 * (int64_t)g.n_real)) return RD_ERR_CUDA;
    auto kern = rd_stream_kernel<MODEL, S>;
    {
        rd_status ast = smem_attr(kern, (int)SS::SMEM);
        if (ast) return ast;
    }
    dim3 grid((unsigned)((g.G + ST_TX - 1) / ST_TX), (unsigned)((g.G + ST_TY - 1) / ST_TY), (unsigned)g.n_real);
    kern<<<grid, ST_THREADS, SS::SMEM, s>>>(tm, dst, g.G, nst, cf, in_dev, out_dev, status);
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL>
static rd_status stream_run(const Handle &h, const GroupDev &g, float *fields, int64_t steps, double *residual,
                            cudaStream_t s) {
    const CoefF cf = make_coef(g);
    const int S = h.stream_depth;
    float *A = fields + g.field_offset, *B = h.d_stream_tmp;
    const int64_t L = steps <= 0 ? 0 : (steps + S - 1) / S;
    for (int64_t k = 0; k < L; ++k) {
        const float *src = (k & 1) ? B : A;
        float *dst = (k & 1) ? A : B;
        const int nst = (int)std::min<int64_t>(S, steps - k * S);
        const int in_dev = k > 0, out_dev = k < L - 1;
        rd_status st;
        switch (S) {
            case 1: st = stream_launch<MODEL, 1>(src, dst, g, nst, cf, in_dev, out_dev, h.d_status, s); break;
            case 2: st = stream_launch<MODEL, 2>(src, dst, g, nst, cf, in_dev, out_dev, h.d_status, s); break;
            case 8: st = stream_launch<MODEL, 8>(src, dst, g, nst, cf, in_dev, out_dev, h.d_status, s); break;
            default: st = stream_launch<MODEL, 4>(src, dst, g, nst, cf, in_dev, out_dev, h.d_status, s); break;
        }
        if (st) return st;
    }
    if (L & 1)
        RD_CUDA_TRY(cudaMemcpyAsync(A, B, sizeof(float) * 2 * (size_t)g.n_real * g.G * g.G, cudaMemcpyDeviceToDevice,
                                    s));
    if (residual) {
        dim3 gp(ST_PARTS, (unsigned)g.n_real);
        stream_residual_part_kernel<MODEL><<<gp, 256, 0, s>>>(A, g.G, g.p[0], g.p[1], g.p[2], g.p[3],
                                                              h.d_stream_part, h.d_status);
        note_launch();
        stream_residual_final_kernel<<<(unsigned)((g.n_real + 127) / 128), 128, 0, s>>>(
            h.d_stream_part, g.n_real, g.G, residual + 2 * g.real_base);
        note_launch();
    }
    return cuda_status(cudaGetLastError());
}

rd_status launch_stream_group(const Handle &h, const GroupDev &g, float *fields, int64_t steps, double *residual,
                              cudaStream_t s) {
    if (!h.d_stream_tmp || !h.d_stream_part) return RD_ERR_INVALID_ARG;
    switch (g.model) {
        case RD_FHN: return stream_run<RD_FHN>(h, g, fields, steps, residual, s);
        case RD_GM: return stream_run<RD_GM>(h, g, fields, steps, residual, s);
        case RD_BZ: return stream_run<RD_BZ>(h, g, fields, steps, residual, s);
        case RD_DIFF: return stream_run<RD_DIFF>(h, g, fields, steps, residual, s);
        default: return RD_ERR_UNSUPPORTED;
    }
}

rd_status stream_reserve(Handle &h) {
    size_t tmp = 0, part = 0;
    for (int i = 0; i < h.n_groups; ++i) {
        const GroupDev &g = h.h_groups[i];
        if (group_is_resident(g) || g.model == RD_RDODE) continue;
        tmp = std::max(tmp, (size_t)2 * g.n_real * g.G * g.G);
        part = std::max(part, (size_t)2 * ST_PARTS * g.n_real);
    }
    h.d_stream_tmp = nullptr;
    h.d_stream_part = nullptr;
    if (h.stream_depth == 0) h.stream_depth = 4;
    if (!tmp) return RD_OK;
    if (cudaMalloc(&h.d_stream_tmp, tmp * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h.d_stream_part, part * sizeof(double)) != cudaSuccess)
        return RD_ERR_OOM;
    return RD_OK;
}

void stream_release(Handle &h) {
    if (h.d_stream_tmp) cudaFree(h.d_stream_tmp);
    if (h.d_stream_part) cudaFree(h.d_stream_part);
    h.d_stream_tmp = nullptr;
    h.d_stream_part = nullptr;
}

}  // namespace rdcil
