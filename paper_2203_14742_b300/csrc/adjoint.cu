// Adjoint of the FP32 explicit Euler stepper: gradient of a sigmoid-smoothed
// correlation integral with respect to the four parameters of one group.
//
// The paper samples with gradient-free methods (DE and adaptive MCMC,
// Sec. 2.1-2.2); this gradient only informs proposals, the likelihood keeps
// the exact indicator counts of eq. (eCDF).
//
//   C_k = (1/(n1 n2)) sum_ij sigma((R_k - d_ij)/tau_k),  tau_k = tau_frac R_k
//   L   = sum_k cot_k C_k
//   lambda_N = dL/dw_N,
//   lambda_n = lambda_{n+1} + dt J_F(w_n)^T lambda_{n+1},
//   g       += dt (dF/dtheta(w_n))^T lambda_{n+1}            (n = N-1 .. 0)
//
// Memory: sqrt(N) checkpointing.  The forward pass stores the state every
// C = ceil(sqrt(N)) steps; the reverse pass recomputes one segment at a time
// into a trajectory buffer (C states) and sweeps it backwards.  The
// Laplacian with mirrored ghosts is symmetric, so
//   sum_cells lambda_u * Lap(u) = sum_cells u * Lap(lambda_u)
// and the diffusion-coefficient gradients need only the halo of lambda.
#include <cmath>
#include <vector>
#include "tile.cuh"

namespace rdcil {

// The reverse sweep records segment q (re-integrating it from its
// checkpoint into a trajectory buffer) on an auxiliary stream while the main
// stream sweeps an earlier-recorded segment backwards; ADJ_NB trajectory
// buffers let the recordings, which depend only on their checkpoints, run
// ahead (events order each buffer's reuse after its reverse sweep).
static constexpr int ADJ_NB = 3;

struct AdjScratch {
    float *ckpt = nullptr;    // [n_seg][n_real][2G^2]
    float *traj = nullptr;    // [ADJ_NB][n_real][C][2G^2]
    float *cur = nullptr;     // [1 + ADJ_NB][n_real][2G^2]: the forward pass, then one per buffer
    float *lam = nullptr;     // [n_real][2G^2]
    double *W = nullptr;      // [n1][n2]
    double *Cbuf = nullptr;   // [32]
    int32_t *sets = nullptr;  // [n1 + n2]
    int32_t *active = nullptr;  // [n_real] realisation appears in a set
    size_t ckpt_f = 0, traj_f = 0, cur_f = 0, W_d = 0, sets_n = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, rec[ADJ_NB] = {}, rev[ADJ_NB] = {};
};

rd_status adjoint_reserve(Handle &h) {
    size_t ck = 0, tr = 0, cu = 0, wd = 0, sn = 0;
    for (int i = 0; i < h.n_groups; ++i) {
        const GroupDev &g = h.h_groups[i];
        if (!(g.flags & RD_GROUP_ADJOINT)) continue;
        int64_t N = g.n_steps < 1 ? 1 : g.n_steps;
        int64_t C = (int64_t)std::ceil(std::sqrt((double)N));
        int64_t nseg = (N + C - 1) / C;
        size_t m = (size_t)g.n_real * 2 * g.G * g.G;
        ck = std::max(ck, (size_t)nseg * m);
        tr = std::max(tr, (size_t)C * m);
        cu = std::max(cu, m);
        wd = std::max(wd, (size_t)g.n_real * g.n_real);
        sn = std::max(sn, (size_t)2 * g.n_real);
    }
    if (!ck) { h.plan = nullptr; return RD_OK; }
    AdjScratch *a = new AdjScratch();
    a->ckpt_f = ck; a->traj_f = tr; a->cur_f = cu; a->W_d = wd; a->sets_n = sn;
    bool ok = cudaMalloc(&a->ckpt, ck * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a->traj, (size_t)ADJ_NB * tr * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a->cur, (size_t)(1 + ADJ_NB) * cu * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a->lam, cu * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a->W, wd * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&a->Cbuf, 32 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&a->sets, sn * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&a->active, (sn / 2 + 1) * sizeof(int32_t)) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&a->aux, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&a->join, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < ADJ_NB && ok; ++b)
        ok = cudaEventCreateWithFlags(&a->rec[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&a->rev[b], cudaEventDisableTiming) == cudaSuccess;
    h.plan = a;
    return ok ? RD_OK : RD_ERR_OOM;
}

void adjoint_release(Handle &h) {
    AdjScratch *a = (AdjScratch *)h.plan;
    if (!a) return;
    cudaFree(a->ckpt); cudaFree(a->traj); cudaFree(a->cur); cudaFree(a->lam);
    cudaFree(a->W); cudaFree(a->Cbuf); cudaFree(a->sets); cudaFree(a->active);
    for (int b = 0; b < ADJ_NB; ++b) {
        if (a->rec[b]) cudaEventDestroy(a->rec[b]);
        if (a->rev[b]) cudaEventDestroy(a->rev[b]);
    }
    if (a->fork) cudaEventDestroy(a->fork);
    if (a->join) cudaEventDestroy(a->join);
    if (a->aux) cudaStreamDestroy(a->aux);
    delete a;
    h.plan = nullptr;
}

// ---------------------------------------------------------------------------
// smoothed correlation integral and dL/dd_ij / d_ij
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t pat_off(int64_t t, int64_t cells, int mask) {
    // component t of the pattern -> offset inside [2][G][G]
    if (mask == 3) return t;
    return (mask == 2 ? cells : 0) + t;
}

__global__ void smooth_fwd_kernel(const float *__restrict__ w, int64_t cells, int mask,
                                  const int32_t *__restrict__ set1, const int32_t *__restrict__ set2, int n1,
                                  int n2, const double *__restrict__ radii, int M, double tau_frac,
                                  const double *__restrict__ cot, double *__restrict__ Cout,
                                  double *__restrict__ W) {
    const int i = blockIdx.y, j = blockIdx.x;
    const int64_t d = (mask == 3 ? 2 : 1) * cells;
    const float *x = w + (int64_t)set1[i] * 2 * cells;
    const float *y = w + (int64_t)set2[j] * 2 * cells;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        int64_t o = pat_off(t, cells, mask);
        double df = (double)x[o] - (double)y[o];
        s += df * df;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double d2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) d2 += red[k];
        double dd = sqrt(d2);
        double inv = 1.0 / ((double)n1 * (double)n2);
        double wsum = 0.0;
        for (int k = 0; k < M; ++k) {
            double tau = tau_frac * radii[k];
            double z = (radii[k] - dd) / tau;
            double sg = 1.0 / (1.0 + exp(-z));
            atomicAdd(&Cout[k], sg * inv);
            if (cot) wsum += cot[k] * (-(sg * (1.0 - sg)) / tau) * inv;
        }
        if (cot) W[(int64_t)i * n2 + j] = dd > 0.0 ? wsum / dd : 0.0;
    }
}

// lambda_N: d L / d pattern, scattered into the state layout.
__global__ void lam_init_kernel(const float *__restrict__ w, int64_t cells, int mask,
                                const int32_t *__restrict__ set1, const int32_t *__restrict__ set2, int n1,
                                int n2, const double *__restrict__ W, float *__restrict__ lam) {
    const int m = blockIdx.x;
    const int64_t d = (mask == 3 ? 2 : 1) * cells;
    const bool first = m < n1;
    const int me = first ? m : m - n1;
    const int r = first ? set1[me] : set2[me];
    const float *xm = w + (int64_t)r * 2 * cells;
    const int nother = first ? n2 : n1;
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        int64_t o = pat_off(t, cells, mask);
        double acc = 0.0;
        double xv = (double)xm[o];
        for (int q = 0; q < nother; ++q) {
            int ro = first ? set2[q] : set1[q];
            double wq = first ? W[(int64_t)me * n2 + q] : W[(int64_t)q * n2 + me];
            double yv = (double)w[(int64_t)ro * 2 * cells + o];
            acc += wq * (xv - yv);   // d d_ij / d x_i = (x_i - x_j)/d_ij, sign flips for set 2
        }
        atomicAdd(&lam[(int64_t)r * 2 * cells + o], (float)acc);
    }
}

// ---------------------------------------------------------------------------
// resident reverse sweep over one segment
// ---------------------------------------------------------------------------
struct AdjCoef {
    float cu, cv, k1, k2, k3;
    double sc[4];   // final scale of the four raw sums
};

template <int MODEL>
__device__ __forceinline__ void adj_cell(float u, float v, float lu, float lv, float Llu, float Llv,
                                         const AdjCoef &c, float &lun, float &lvn, float (&s)[4]) {
    s[0] = fmaf(u, Llu, s[0]);
    s[1] = fmaf(v, Llv, s[1]);
    if (MODEL == RD_FHN) {
        // J^T: [1-3u^2, eps; -1, -eps a]
        float a = fmaf(-3.f * u, u, 1.f);
        lun = fmaf(c.cu, Llu, fmaf(c.k1 * a, lu, fmaf(c.k2, lv, lu)));
        lvn = fmaf(c.cv, Llv, fmaf(-c.k1, lu, fmaf(-c.k2 * c.k3, lv, lv)));
        s[2] = fmaf(fmaf(-c.k3, v, u), lv, s[2]);    // (u - a v) lambda_v
        s[3] = fmaf(v, lv, s[3]);                    // v lambda_v   (x -eps dt)
    } else if (MODEL == RD_GM) {
        // J^T: rho [2u/v - mu, 2u; -u^2/v^2, -1]
        float iv = __fdividef(1.f, v);
        float q = u * iv;
        lun = fmaf(c.cu, Llu, fmaf(c.k2, fmaf(fmaf(2.f, q, -c.k3), lu, 2.f * u * lv), lu));
        lvn = fmaf(c.cv, Llv, fmaf(c.k2, fmaf(-q * q, lu, -lv), lv));
        s[2] = fmaf(fmaf(u, q, -c.k3 * u), lu, fmaf(fmaf(u, u, -v), lv, s[2]));
        s[3] = fmaf(u, lu, s[3]);                    // u lambda_u   (x -rho dt)
    } else if (MODEL == RD_BZ) {
        // J^T: [2uv - (B+1), B - 2uv; u^2, -u^2]; with dl = lambda_u - lambda_v
        // the u row is (2uv - B) dl - lambda_u and the v row u^2 dl
        const float dl = lu - lv;
        const float t = fmaf(2.f * u, v, -c.k3);
        lun = fmaf(c.cu, Llu, fmaf(c.k1, fmaf(t, dl, -lu), lu));
        lvn = fmaf(c.cv, Llv, fmaf(c.k1, (u * u) * dl, lv));
        s[2] = s[2] + lu;                            // dF/dA = (1, 0)       (x dt)
        s[3] = fmaf(-u, dl, s[3]);                   // dF/dB = (-u, u)      (x dt)
    } else {
        lun = fmaf(c.cu, Llu, lu);
        lvn = fmaf(c.cv, Llv, lv);
    }
}

template <int MODEL, int G, int TY, int TX>
__global__ void __launch_bounds__(Tiling<G, TY, TX>::NT, 1)
rd_adjoint_reverse_kernel(const float *__restrict__ traj, int64_t traj_stride, int64_t len,
                          float *__restrict__ lam, AdjCoef cf, double *__restrict__ gacc,
                          const int32_t *__restrict__ active) {
    using T = Tiling<G, TY, TX>;
    constexpr int NX = T::NX;
    extern __shared__ float4 smem_f4[];
    float *sm = reinterpret_cast<float *>(smem_f4);
    const int tid = threadIdx.x, tx = tid % NX, ty = tid / NX;
    const int r = blockIdx.x;
    if (!active[r]) return;   // realisation outside both sets: lambda stays 0
    float *lbase = lam + (int64_t)r * 2 * G * G;
    float lu[TY][TX], lv[TY][TX];
    tile_load<G, TY, TX>(lbase, tx, ty, lu, lv);
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    // the state of step n is loaded one step ahead (un, vn), so its global
    // loads overlap the previous step's arithmetic
    const float *tr = traj + (int64_t)r * traj_stride;
    float un[TY][TX], vn[TY][TX];
    if (len > 0) tile_load<G, TY, TX>(tr + (len - 1) * 2 * G * G, tx, ty, un, vn);
    for (int64_t n = len - 1; n >= 0; --n) {
        float u[TY][TX], v[TY][TX];
#pragma unroll
        for (int i = 0; i < TY; ++i)
#pragma unroll
            for (int c = 0; c < TX; ++c) { u[i][c] = un[i][c]; v[i][c] = vn[i][c]; }
        if (n > 0) tile_load<G, TY, TX>(tr + (n - 1) * 2 * G * G, tx, ty, un, vn);
        float *hb = sm + (int)(n & 1) * (T::HALO_FLOATS / 2);
        halo_put<G, TY, TX>(hb, tx, ty, lu, lv);
        __syncthreads();
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        float pu[TX], pv[TX];
        halo_north<G, TY, TX>(hb, tx, ty, lu, lv, pu, pv);
#pragma unroll
        for (int i = 0; i < TY; ++i) {
            float su[TX], sv[TX];
            row_south<G, TY, TX>(hb, tx, ty, i, lu, lv, su, sv);
            float wu, eu, wv, ev;
            row_west_east<NX>(tx, lu[i][0], lu[i][TX - 1], wu, eu);
            row_west_east<NX>(tx, lv[i][0], lv[i][TX - 1], wv, ev);
            float cu_[TX], cv_[TX];
#pragma unroll
            for (int c = 0; c < TX; ++c) { cu_[c] = lu[i][c]; cv_[c] = lv[i][c]; }
#pragma unroll
            for (int c = 0; c < TX; ++c) {
                float Wu = c > 0 ? cu_[c - 1] : wu, Eu = c < TX - 1 ? cu_[c + 1] : eu;
                float Wv = c > 0 ? cv_[c - 1] : wv, Ev = c < TX - 1 ? cv_[c + 1] : ev;
                float Llu = fmaf(-4.f, cu_[c], (pu[c] + su[c]) + (Wu + Eu));
                float Llv = fmaf(-4.f, cv_[c], (pv[c] + sv[c]) + (Wv + Ev));
                adj_cell<MODEL>(u[i][c], v[i][c], cu_[c], cv_[c], Llu, Llv, cf, lu[i][c], lv[i][c], s);
            }
#pragma unroll
            for (int c = 0; c < TX; ++c) { pu[c] = cu_[c]; pv[c] = cv_[c]; }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] += (double)s[k];
    }
    tile_store<G, TY, TX>(lbase, tx, ty, lu, lv);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g[k] += __shfl_xor_sync(0xffffffffu, g[k], o);
    }
    __syncthreads();
    double *red = reinterpret_cast<double *>(sm);
    constexpr int NW = T::NT / 32;
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k * NW + warp] = g[k];
    __syncthreads();
    if (tid < 4) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += red[tid * NW + w];
        atomicAdd(&gacc[tid], s * cf.sc[tid]);
    }
}

template <int G> struct AdjTile;
template <> struct AdjTile<32> { static constexpr int TY = 4, TX = 4; };
template <> struct AdjTile<64> { static constexpr int TY = 4, TX = 4; };
template <> struct AdjTile<128> { static constexpr int TY = 8, TX = 4; };

template <int MODEL, int G>
static rd_status launch_reverse(const GroupDev &g, const float *traj, int64_t traj_stride, int64_t len, float *lam,
                                const AdjCoef &cf, double *gacc, const int32_t *active, cudaStream_t s) {
    constexpr int TY = AdjTile<G>::TY, TX = AdjTile<G>::TX;
    using T = Tiling<G, TY, TX>;
    auto kern = rd_adjoint_reverse_kernel<MODEL, G, TY, TX>;
    {
        rd_status ast = smem_attr(kern, (int)T::SMEM);
        if (ast) return ast;
    }
    kern<<<g.n_real, T::NT, T::SMEM, s>>>(traj, traj_stride, len, lam, cf, gacc, active);
    note_launch();
    return cuda_status(cudaGetLastError());
}

template <int MODEL>
static rd_status reverse_G(const GroupDev &g, const float *traj, int64_t ts, int64_t len, float *lam,
                           const AdjCoef &cf, double *gacc, const int32_t *active, cudaStream_t s) {
    switch (g.G) {
        case 32: return launch_reverse<MODEL, 32>(g, traj, ts, len, lam, cf, gacc, active, s);
        case 64: return launch_reverse<MODEL, 64>(g, traj, ts, len, lam, cf, gacc, active, s);
        case 128: return launch_reverse<MODEL, 128>(g, traj, ts, len, lam, cf, gacc, active, s);
        default: return RD_ERR_UNSUPPORTED;
    }
}

__global__ void mark_active_kernel(const int32_t *__restrict__ sets, int n, int32_t *__restrict__ active) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) active[sets[q]] = 1;
}

}  // namespace rdcil

using namespace rdcil;

extern "C" rd_status rd_adjoint(rd_handle *hh, int32_t group, const float *d_fields0, int32_t species_mask,
                                const int32_t *set1, int64_t n1, const int32_t *set2, int64_t n2,
                                const double *d_radii, int32_t M, double tau_frac, const double *d_cotangent,
                                double *d_C, double *d_grad, void *stream) {
    if (!hh || !d_fields0 || !set1 || !set2 || !d_radii) return RD_ERR_INVALID_ARG;
    // forward only (C, no gradient) when neither cotangent nor gradient is given
    const bool fwd_only = !d_cotangent && !d_grad;
    if (!fwd_only && (!d_cotangent || !d_grad)) return RD_ERR_INVALID_ARG;
    if (fwd_only && !d_C) return RD_ERR_INVALID_ARG;
    Handle &h = *reinterpret_cast<Handle *>(hh);
    if (group < 0 || group >= h.n_groups) return RD_ERR_INVALID_ARG;
    const GroupDev &g = h.h_groups[group];
    if (!(g.flags & RD_GROUP_ADJOINT) || !h.plan) return RD_ERR_INVALID_ARG;
    if (species_mask < 1 || species_mask > 3 || M < 1 || M > 32 || !(tau_frac > 0.0)) return RD_ERR_INVALID_ARG;
    if (n1 < 1 || n2 < 1 || n1 > g.n_real || n2 > g.n_real) return RD_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n1; ++i)
        if (set1[i] < 0 || set1[i] >= g.n_real) return RD_ERR_INVALID_ARG;
    for (int64_t j = 0; j < n2; ++j)
        if (set2[j] < 0 || set2[j] >= g.n_real) return RD_ERR_INVALID_ARG;
    AdjScratch &a = *(AdjScratch *)h.plan;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t cells = (int64_t)g.G * g.G, m = 2 * cells, mall = m * g.n_real;
    const int64_t N = g.n_steps;
    const int64_t C = N < 1 ? 1 : (int64_t)std::ceil(std::sqrt((double)N));
    const int64_t nseg = N < 1 ? 0 : (N + C - 1) / C;

    // stage the index sets (host -> device, through the stream)
    std::vector<int32_t> sets((size_t)(n1 + n2));
    for (int64_t i = 0; i < n1; ++i) sets[i] = set1[i];
    for (int64_t j = 0; j < n2; ++j) sets[n1 + j] = set2[j];
    RD_CUDA_TRY(cudaMemcpyAsync(a.sets, sets.data(), sets.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int32_t *d_s1 = a.sets, *d_s2 = a.sets + n1;

    // forward with checkpoints
    GroupDev gl = g;
    gl.field_offset = 0;
    gl.real_base = 0;
    RD_CUDA_TRY(cudaMemcpyAsync(a.cur, d_fields0 + g.field_offset, mall * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (fwd_only) {
        if (N > 0) {
            rd_status st = launch_integrate_group(gl, a.cur, N, nullptr, h.d_status, s);
            if (st) return st;
        }
        RD_CUDA_TRY(cudaMemsetAsync(d_C, 0, M * sizeof(double), s));
        dim3 gp((unsigned)n2, (unsigned)n1);
        smooth_fwd_kernel<<<gp, 256, 0, s>>>(a.cur, cells, species_mask, d_s1, d_s2, (int)n1, (int)n2, d_radii, M,
                                             tau_frac, nullptr, d_C, a.W);
        note_launch();
        return cuda_status(cudaGetLastError());
    }
    for (int64_t q = 0; q < nseg; ++q) {
        int64_t len = std::min(C, N - q * C);
        RD_CUDA_TRY(cudaMemcpyAsync(a.ckpt + q * mall, a.cur, mall * sizeof(float), cudaMemcpyDeviceToDevice, s));
        rd_status st = launch_integrate_group(gl, a.cur, len, nullptr, h.d_status, s);
        if (st) return st;
    }
    // smoothed CIL and lambda_N
    double *Cout = d_C ? d_C : a.Cbuf;
    RD_CUDA_TRY(cudaMemsetAsync(Cout, 0, M * sizeof(double), s));
    RD_CUDA_TRY(cudaMemsetAsync(a.lam, 0, mall * sizeof(float), s));
    RD_CUDA_TRY(cudaMemsetAsync(d_grad, 0, 4 * sizeof(double), s));
    dim3 gp((unsigned)n2, (unsigned)n1);
    smooth_fwd_kernel<<<gp, 256, 0, s>>>(a.cur, cells, species_mask, d_s1, d_s2, (int)n1, (int)n2, d_radii, M,
                                         tau_frac, d_cotangent, Cout, a.W);
    note_launch();
    lam_init_kernel<<<(unsigned)(n1 + n2), 256, 0, s>>>(a.cur, cells, species_mask, d_s1, d_s2, (int)n1, (int)n2,
                                                        a.W, a.lam);
    note_launch();
    // realisations that appear in a set (others keep lambda = 0 and are skipped)
    int32_t *active = a.active;
    RD_CUDA_TRY(cudaMemsetAsync(active, 0, g.n_real * sizeof(int32_t), s));
    mark_active_kernel<<<1, 256, 0, s>>>(a.sets, (int)(n1 + n2), active);
    note_launch();
    RD_CUDA_TRY(cudaGetLastError());

    // reverse sweep
    AdjCoef cf;
    CoefF f = make_coef(g);
    cf.cu = f.cu; cf.cv = f.cv; cf.k1 = f.k1; cf.k2 = f.k2; cf.k3 = f.k3;
    const double h2 = (double)(g.G - 1) * (double)(g.G - 1);
    cf.sc[0] = g.dt * h2;
    cf.sc[1] = g.dt * h2;
    if (g.model == RD_FHN) { cf.sc[2] = g.dt; cf.sc[3] = -g.p[2] * g.dt; }
    else if (g.model == RD_GM) { cf.sc[2] = g.dt; cf.sc[3] = -g.p[2] * g.dt; }
    else if (g.model == RD_BZ) { cf.sc[2] = g.dt; cf.sc[3] = g.dt; }
    else { cf.sc[2] = 0.0; cf.sc[3] = 0.0; }
    // recordings on the auxiliary stream (after everything above), reverse
    // sweeps on s, buffer b = k mod ADJ_NB for the k-th segment from the end
    RD_CUDA_TRY(cudaEventRecord(a.fork, s));
    RD_CUDA_TRY(cudaStreamWaitEvent(a.aux, a.fork, 0));
    const size_t trb = a.traj_f;   // floats per trajectory buffer
    int64_t k = 0;
    for (int64_t q = nseg - 1; q >= 0; --q, ++k) {
        const int b = (int)(k % ADJ_NB);
        const int64_t len = std::min(C, N - q * C);
        float *traj = a.traj + (size_t)b * trb, *cur = a.cur + (size_t)(1 + b) * a.cur_f;
        if (k >= ADJ_NB) RD_CUDA_TRY(cudaStreamWaitEvent(a.aux, a.rev[b], 0));   // the buffer's last sweep done
        RD_CUDA_TRY(cudaMemcpyAsync(cur, a.ckpt + q * mall, mall * sizeof(float), cudaMemcpyDeviceToDevice, a.aux));
        rd_status st = launch_record_group(gl, cur, traj, len, a.aux);
        if (st) return st;
        RD_CUDA_TRY(cudaEventRecord(a.rec[b], a.aux));
        RD_CUDA_TRY(cudaStreamWaitEvent(s, a.rec[b], 0));
        const int64_t ts = len * m;
        switch (g.model) {
            case RD_FHN: st = reverse_G<RD_FHN>(g, traj, ts, len, a.lam, cf, d_grad, active, s); break;
            case RD_GM: st = reverse_G<RD_GM>(g, traj, ts, len, a.lam, cf, d_grad, active, s); break;
            case RD_BZ: st = reverse_G<RD_BZ>(g, traj, ts, len, a.lam, cf, d_grad, active, s); break;
            default: st = reverse_G<RD_DIFF>(g, traj, ts, len, a.lam, cf, d_grad, active, s); break;
        }
        if (st) return st;
        RD_CUDA_TRY(cudaEventRecord(a.rev[b], s));
    }
    RD_CUDA_TRY(cudaEventRecord(a.join, a.aux));
    RD_CUDA_TRY(cudaStreamWaitEvent(s, a.join, 0));
    return RD_OK;
}
