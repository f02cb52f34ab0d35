// Multi-feature correlation integral (MCIL): the correlation integral
// vector of eq. (CIL) under six distances of the pattern difference
// u = s_i - s_j, concatenated (Sec. 3.1, Alg. 2), optionally on min-max
// scaled patterns (Sec. 4, "scaled pattern data").
//
// A pattern is n_species fields of Gy x Gx nodes (Gy = Gx = G for the 2-D
// models, Gy = 1 for the 1-D reaction-diffusion-ODE patterns, which have no
// y differences: qy = my = 0); h = 1/(Gx-1), g = Gx-1.  The derivative
// patterns are forward differences of each field rounded to FP32 once
// (Dx: Gy x (Gx-1), Dy: (Gy-1) x Gx per species).  With q0, qx, qy the
// squared distances of the CIL (the exact real sum of squared differences,
// rounded once to the nearest double) of the patterns and of their Dx and
// Dy patterns,
// and m0, mx, my the maxima of |difference| with each difference in FP64
// (rounded to nearest, like the squared distance's), the features are
//   0 L2      squared  q0                                  (eq. norm:L2)
//   1 Linf    value    m0                                  (eq. norm:Linf)
//   2 W12     squared  (h^2 q0 + qx) + qy                  (eq. norm:W12)
//   3 W12'    value    (h sqrt(q0) + sqrt(qx)) + sqrt(qy)   (eq. norm:W12prime)
//   4 W1inf   value    max(m0, max(g mx, g my))            (eq. norm:W1inf)
//   5 W1inf'  value    (m0 + g mx) + g my                  (eq. norm:W1infprime)
// each one FP64 expression with every operation rounded to nearest.  A
// squared feature is decided like the CIL (R0 = sqrt(max), V < R_k * R_k),
// a value feature directly (R0 = max, V < R_k); R_k = R_{k-1} / b (power
// law) or R_k = R0 - k (R0 - R_min) / M with R_min the smallest value (its
// sqrt for a squared feature; the linear law of Sec. 2.1 / Sec. 3.2).
//
// Exactness contract: bins and counts equal that definition bit for bit.
//   1. q0, qx, qy: tier-1 intervals of the CIL (centred bf16 hi/lo split,
//      tensor-core Gram, rigorous bound), one run per pattern array;
//   2. m0, mx, my: a tiled SIMT pass (split over K, partial maxima met by
//      atomicMax) takes max |fl32(a - b)|; rounding to nearest is monotone,
//      so that is fl32 of the exact maximum M, and M (and its FP64 rounding,
//      the defined value) lies within m32 (1 -+ 2^-23);
//   3. per pair and feature, an FP64 interval of the feature value by
//      outward-rounded (_rd / _ru) evaluation of its expression (every
//      operation is monotone on the non-negative inputs);
//   4. pairs whose interval may hold a feature's maximum (linear law: or
//      its minimum) are evaluated exactly (integer fixed-point sums rounded
//      once, exact.cuh; one CTA per pair and pattern array), which fixes R0
//      (and R_min) and the radii; pairs whose interval meets a threshold
//      get tier 2 (FP32 error-free squared distances with a ~1e-12 bound,
//      exact maxima) and, if still undecided, the exact evaluation; every
//      other pair is decided by its interval.
#include <cuda_runtime.h>
#include "common.cuh"
#include "exact.cuh"
#include "tma.cuh"

rd_status cil_tier1_intervals(const float *X1, int64_t ld1, int64_t n1, const float *X2, int64_t ld2, int64_t n2,
                              int64_t d, void *work, size_t work_bytes, const float **lo, const float **hi,
                              const unsigned long long **timeout, cudaStream_t s);
extern "C" rd_status cil_workspace_size(int64_t n1, int64_t n2, int64_t d, size_t *bytes);

namespace rdcil {

static constexpr int NF = 6;
static constexpr int MC_SCAL = 32;   // control words of one call (see McilWork::scal)
static constexpr int EX_CAP = 4096;  // queued pairs the split exact evaluation takes per launch
__host__ __device__ constexpr bool feat_squared(int f) { return f == 0 || f == 2; }

struct McilWork {
    int64_t n1, n2, np, d0, dex, dey;
    int Gy, Gx, nsp, mask, M, law;   // law 0 power, 1 linear, 2 fitted power (1 and 2 need the minima),
                                     // 3 given radii (no maxima or minima needed)
    float *S1, *S2;                 // min-max scaled patterns (scale only)
    float *Ax1, *Ay1, *Ax2, *Ay2;   // forward-difference patterns
    void *cw[3];                    // CIL workspaces for the pattern, Dx, Dy arrays
    size_t cw_bytes[3];
    float *mabs;                    // [3][np] FP32 max |difference| of the three arrays
    double *vlo, *vhi;              // [NF][np] feature intervals
    double *vex;                    // [NF][np] exact feature values (where flag == 2)
    uint8_t *flag;                  // [np] 0 interval, 1 queued, 2 exact
    int64_t *queue;                 // [np] pairs to evaluate exactly
    unsigned long long *scal;       // [0] queue length; [1] end of the maximum-candidate phase; [2 + f]
                                    // largest lower bound of feature f (bits); [8] start of the final
                                    // exact segment; [9] number of maximum candidates; [10] pairs
                                    // evaluated exactly; [16 + f] smallest upper
                                    // bound of feature f (complemented bits, linear law)
    double *thr;                    // [NF][32] thresholds of the decision (R_k^2 or R_k)
    double *grp;                    // [EX_CAP][3][2] exact squared distance and maximum per array
    unsigned int *arrive;           // [EX_CAP] arrays finished per queued pair
    size_t bytes;
};

static inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

static McilWork mlayout(int64_t n1, int64_t n2, int Gy, int Gx, int nsp, int mask, int scale, int M, void *base) {
    McilWork w{};
    w.n1 = n1; w.n2 = n2; w.np = n1 * n2; w.Gy = Gy; w.Gx = Gx; w.nsp = nsp; w.mask = mask; w.M = M;
    w.d0 = (int64_t)nsp * Gy * Gx;
    w.dex = (int64_t)nsp * Gy * (Gx - 1);
    w.dey = (int64_t)nsp * (Gy - 1) * Gx;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)rup((int64_t)(off + bytes), 256);
        return (char *)base + o;
    };
    const int64_t n = n1 + n2;
    if (scale) {
        w.S1 = (float *)take(sizeof(float) * n1 * w.d0);
        w.S2 = (float *)take(sizeof(float) * n2 * w.d0);
    }
    const bool deriv = (mask & 0x3C) != 0;
    if (deriv) {
        w.Ax1 = (float *)take(sizeof(float) * n1 * w.dex);
        w.Ax2 = (float *)take(sizeof(float) * n2 * w.dex);
        if (w.dey > 0) {
            w.Ay1 = (float *)take(sizeof(float) * n1 * w.dey);
            w.Ay2 = (float *)take(sizeof(float) * n2 * w.dey);
        }
    }
    (void)n;
    const bool need_q0 = (mask & 0x0D) != 0, need_qd = (mask & 0x0C) != 0;
    for (int a = 0; a < 3; ++a) {
        const int64_t da = a == 0 ? w.d0 : (a == 1 ? w.dex : w.dey);
        const bool need = (a == 0 ? need_q0 : need_qd) && da > 0;
        w.cw[a] = nullptr;
        w.cw_bytes[a] = 0;
        if (need) {
            size_t sz = 0;
            cil_workspace_size(n1, n2, da, &sz);
            w.cw_bytes[a] = sz;
            w.cw[a] = take(sz);
        }
    }
    w.mabs = (float *)take(sizeof(float) * 3 * w.np);
    w.vlo = (double *)take(sizeof(double) * NF * w.np);
    w.vhi = (double *)take(sizeof(double) * NF * w.np);
    w.vex = (double *)take(sizeof(double) * NF * w.np);
    w.flag = (uint8_t *)take(w.np);
    w.queue = (int64_t *)take(sizeof(int64_t) * w.np);
    w.scal = (unsigned long long *)take(sizeof(unsigned long long) * MC_SCAL);
    w.thr = (double *)take(sizeof(double) * NF * 32);
    w.grp = (double *)take(sizeof(double) * EX_CAP * 6);
    w.arrive = (unsigned int *)take(sizeof(unsigned int) * EX_CAP);
    w.bytes = off;
    return w;
}

// ---------------------------------------------------------------------------
// 0. min-max scaling: one CTA per (pattern, species)
// ---------------------------------------------------------------------------
__global__ void minmax_kernel(const float *__restrict__ X, int64_t ld, int64_t cells, int nsp,
                              float *__restrict__ out) {
    const int64_t i = blockIdx.x / nsp;
    const int sp = blockIdx.x % nsp;
    const float *x = X + i * ld + sp * cells;
    float *o = out + (i * nsp + sp) * cells;
    float mn = x[0], mx = x[0];
    for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) {
        mn = fminf(mn, x[c]);
        mx = fmaxf(mx, x[c]);
    }
    __shared__ float smn[32], smx[32];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o2));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { smn[warp] = mn; smx[warp] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) { smn[0] = fminf(smn[0], smn[q]); smx[0] = fmaxf(smx[0], smx[q]); }
    }
    __syncthreads();
    mn = smn[0];
    mx = smx[0];
    const double span = __dsub_rn((double)mx, (double)mn);
    for (int64_t c = threadIdx.x; c < cells; c += blockDim.x)
        o[c] = mx > mn ? __double2float_rn(__ddiv_rn(__dsub_rn((double)x[c], (double)mn), span)) : 0.0f;
}

// ---------------------------------------------------------------------------
// 1. forward-difference patterns (FP32 subtraction = the exact difference
//    rounded once)
// ---------------------------------------------------------------------------
__global__ void fd_kernel(const float *__restrict__ X, int64_t ld, int64_t n, int Gy, int Gx, int nsp,
                          float *__restrict__ Ax, float *__restrict__ Ay) {
    // one grid row r = (pattern i, species sp, row y) at a time; threads
    // along x (coalesced reads of rows y and y + 1)
    const int64_t cex = (int64_t)Gy * (Gx - 1), cey = (int64_t)(Gy - 1) * Gx, cells = (int64_t)Gy * Gx;
    const int64_t nrows = n * nsp * Gy;
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int64_t is = r / Gy;
        const int y = (int)(r - is * Gy);
        const int64_t i = is / nsp;
        const int sp = (int)(is - i * nsp);
        const float *x = X + i * ld + (int64_t)sp * cells + (int64_t)y * Gx;
        float *dx = Ax + is * cex + (int64_t)y * (Gx - 1);
        for (int c = threadIdx.x; c < Gx - 1; c += blockDim.x) dx[c] = x[c + 1] - x[c];
        if (y < Gy - 1) {
            float *dy = Ay + is * cey + (int64_t)y * Gx;
            for (int c = threadIdx.x; c < Gx; c += blockDim.x) dy[c] = x[Gx + c] - x[c];
        }
    }
}

// The same for Gx a multiple of 4 (and at most 128 x 32 = 4096): a warp
// covers up to 128 columns of one row with float4 loads, the column right
// of a lane's four comes from the next lane by shuffle, the next row by a
// float4 load; eight rows (warps) per block, so every block has eight rows'
// loads in flight.  Dx rows (Gx - 1 values) are stored value by value, Dy
// rows as float4.
__global__ void __launch_bounds__(256) fd4_kernel(const float *__restrict__ X, int64_t ld, int64_t n, int Gy,
                                                   int Gx, int nsp, float *__restrict__ Ax, float *__restrict__ Ay) {
    const int64_t cex = (int64_t)Gy * (Gx - 1), cey = (int64_t)(Gy - 1) * Gx, cells = (int64_t)Gy * Gx;
    const int64_t nrows = n * nsp * Gy;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = Gx >> 2;   // float4 per row
    for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < nrows; r += (int64_t)gridDim.x * 8) {
        const int64_t is = r / Gy;
        const int y = (int)(r - is * Gy);
        const int64_t i = is / nsp;
        const int sp = (int)(is - i * nsp);
        const float *x = X + i * ld + (int64_t)sp * cells + (int64_t)y * Gx;
        float *dx = Ax + is * cex + (int64_t)y * (Gx - 1);
        float *dy = (y < Gy - 1) ? Ay + is * cey + (int64_t)y * Gx : nullptr;
        for (int q0 = 0; q0 < nq; q0 += 32) {
            const int q = q0 + lane;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (q < nq) {
                a = *reinterpret_cast<const float4 *>(x + 4 * q);
                if (dy) b = *reinterpret_cast<const float4 *>(x + Gx + 4 * q);
            }
            // first value of the next lane's four (the next 32-float4 slice
            // starts a fresh warp-wide load, read directly)
            float nx = __shfl_down_sync(0xffffffffu, a.x, 1);
            if (lane == 31 && q + 1 < nq) nx = x[4 * (q + 1)];
            if (q < nq) {
                const int c = 4 * q;
                dx[c] = a.y - a.x;
                dx[c + 1] = a.z - a.y;
                dx[c + 2] = a.w - a.z;
                if (c + 3 < Gx - 1) dx[c + 3] = nx - a.w;
                if (dy)
                    *reinterpret_cast<float4 *>(dy + c) = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 2. max |a - b| of every pair, FP32: 128 x 128 (or 64 x 256) pairs per
//    CTA, 8 x 8 per thread, 32-column slices of both sets in shared memory,
//    and a split of K over blockIdx.z whose partial maxima meet in atomicMax
//    on the FP32 bit patterns (non-negative floats order like their bits;
//    max is exact in any order)
// ---------------------------------------------------------------------------
constexpr int MX_K = 32;
// max(|a|, |b|, |c|): the three-input FP32 max with absolute values
__device__ __forceinline__ float max3_abs(float a, float b, float c) {
    float d;
    asm("max.abs.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// TA x TB pairs per CTA (TA = 128 or 64 set-1 rows; TB = 32768 / TA set-2
// rows), 8 x 8 per thread: thread (ty, tx) takes rows ty + (TA/8) a and
// columns tx + (TB/8) c, so the shared-memory reads of a warp are
// broadcasts (rows) or consecutive words (columns)
// Thread (ty, tx) of RY x RX takes set-1 rows a4 * TA/2 + 4 ty + q and set-2
// rows c4 * TB/2 + 4 tx + q (a4, c4 in {0, 1}, q < 4): four consecutive
// rows per 128-bit shared load (broadcast for set 1, 512 contiguous bytes a
// warp for set 2).  Each K column of a tile is a row of TA (TB) floats
// padded by 4 to keep 16-byte alignment.
template <int TA>
struct MaxTile {
    static constexpr int TB = 16384 / TA, RY = TA / 8, RX = TB / 8;   // RY x RX = 256 threads
    static constexpr int PA = TA + 4, PB = TB + 4;                     // padded K-column rows
    static constexpr int SA = MX_K * PA, SB = MX_K * PB;               // floats per buffer
    static constexpr size_t SMEM = 2 * (size_t)(SA + SB) * sizeof(float);   // two buffers
};

// 4-byte asynchronous copy global -> shared; src_bytes = 0 writes a zero
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

template <int TA>
__global__ void __launch_bounds__(256, 2) maxabs_kernel(const float *__restrict__ A, int64_t lda, int64_t n1,
                                                        const float *__restrict__ B, int64_t ldb, int64_t n2,
                                                        int64_t d, int64_t kch, float *__restrict__ out) {
    using MT = MaxTile<TA>;
    constexpr int TB = MT::TB, RY = MT::RY, RX = MT::RX, PA = MT::PA, PB = MT::PB;
    static_assert(RY * RX == 256, "thread grid");
    extern __shared__ float4 mx_smem[];
    float *sm = reinterpret_cast<float *>(mx_smem);
    // buffer q: sa = sm + q (SA + SB), sb = sa + SA; element [kk][r]
    const int64_t i0 = (int64_t)blockIdx.y * TA, j0 = (int64_t)blockIdx.x * TB;
    const int64_t k_lo = (int64_t)blockIdx.z * kch, k_hi = min(d, k_lo + kch);
    const int tx = threadIdx.x % RX, ty = threadIdx.x / RX;
    // K chunk starting at k0 into buffer q (a warp copies 32 consecutive
    // columns of one row)
    auto load = [&](int q, int64_t k0) {
        float *sa = sm + q * (MT::SA + MT::SB), *sb = sa + MT::SA;
        for (int e = threadIdx.x; e < TA * MX_K; e += 256) {
            const int r = e / MX_K, kk = e - r * MX_K;
            const int64_t k = k0 + kk, ia = i0 + r;
            const bool in = ia < n1 && k < k_hi;
            cp_async4(sa + kk * PA + r, in ? A + ia * lda + k : A, in ? 4 : 0);
        }
        for (int e = threadIdx.x; e < TB * MX_K; e += 256) {
            const int r = e / MX_K, kk = e - r * MX_K;
            const int64_t k = k0 + kk, jb = j0 + r;
            const bool in = jb < n2 && k < k_hi;
            cp_async4(sb + kk * PB + r, in ? B + jb * ldb + k : B, in ? 4 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float m[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) m[a][c] = 0.f;
    if (k_lo < k_hi) load(0, k_lo);
    int q = 0;
    for (int64_t k0 = k_lo; k0 < k_hi; k0 += MX_K, q ^= 1) {
        const bool more = k0 + MX_K < k_hi;
        if (more) {
            load(q ^ 1, k0 + MX_K);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float *sa = sm + q * (MT::SA + MT::SB), *sb = sa + MT::SA;
        // two K columns per step: m = max(|m|, |d1|, |d2|) in one three-input
        // max (exact in any grouping; m >= 0)
#pragma unroll 2
        for (int kk = 0; kk < MX_K; kk += 2) {
            float av[8], bv[8], aw[8], bw[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 x0 = *reinterpret_cast<const float4 *>(sa + kk * PA + h * (TA / 2) + 4 * ty);
                const float4 x1 = *reinterpret_cast<const float4 *>(sa + (kk + 1) * PA + h * (TA / 2) + 4 * ty);
                const float4 y0 = *reinterpret_cast<const float4 *>(sb + kk * PB + h * (TB / 2) + 4 * tx);
                const float4 y1 = *reinterpret_cast<const float4 *>(sb + (kk + 1) * PB + h * (TB / 2) + 4 * tx);
                av[4 * h] = x0.x; av[4 * h + 1] = x0.y; av[4 * h + 2] = x0.z; av[4 * h + 3] = x0.w;
                aw[4 * h] = x1.x; aw[4 * h + 1] = x1.y; aw[4 * h + 2] = x1.z; aw[4 * h + 3] = x1.w;
                bv[4 * h] = y0.x; bv[4 * h + 1] = y0.y; bv[4 * h + 2] = y0.z; bv[4 * h + 3] = y0.w;
                bw[4 * h] = y1.x; bw[4 * h + 1] = y1.y; bw[4 * h + 2] = y1.z; bw[4 * h + 3] = y1.w;
            }
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) m[a][c] = max3_abs(m[a][c], av[a] - bv[c], aw[a] - bw[c]);
        }
        __syncthreads();   // buffer q is refilled two chunks on
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t i = i0 + (a >> 2) * (TA / 2) + 4 * ty + (a & 3);
            const int64_t j = j0 + (c >> 2) * (TB / 2) + 4 * tx + (c & 3);
            if (i < n1 && j < n2 && m[a][c] > 0.f)
                atomicMax(reinterpret_cast<unsigned int *>(out) + i * n2 + j, __float_as_uint(m[a][c]));
        }
}

// ---------------------------------------------------------------------------
// 3. feature intervals (outward rounding) and the largest lower bound
// ---------------------------------------------------------------------------
struct QIv {
    const float *lo[3], *hi[3];
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v) {
    atomicMax(a, (unsigned long long)__double_as_longlong(fmax(v, 0.0)));
}
// the minimum through atomicMax on the complemented bits (non-negative
// doubles order like their bits; the cleared word reads as "none yet")
__device__ __forceinline__ void atomic_min_nonneg(unsigned long long *a, double v) {
    atomicMax(a, ~(unsigned long long)__double_as_longlong(fmax(v, 0.0)));
}
__device__ __forceinline__ double read_min_nonneg(const unsigned long long *a) {
    return __longlong_as_double((long long)~*a);
}

__global__ void intervals_kernel(McilWork w, QIv qi, double h, double h2, double g) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t np = w.np;
    double lb[NF], ub[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        lb[f] = 0.0;
        ub[f] = __longlong_as_double(0x7ff0000000000000ll);
    }
    if (q < np) {
        double ql[3] = {0, 0, 0}, qh[3] = {0, 0, 0}, ml[3] = {0, 0, 0}, mh[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (qi.lo[a]) {
                ql[a] = fmax((double)qi.lo[a][q], 0.0);
                qh[a] = fmax((double)qi.hi[a][q], 0.0);
            }
            // |m32 - M| <= 2^-24 M for the exact maximum M, so M lies in
            // [m32 / (1 + 2^-24), m32 / (1 - 2^-24)], inside m32 (1 -+ 2^-23)
            const double m32 = (double)w.mabs[a * np + q];
            ml[a] = __dmul_rd(m32, 1.0 - 1.1920928955078125e-7);
            mh[a] = __dmul_ru(m32, 1.0 + 1.1920928955078125e-7);
        }
        double lo[NF], hi[NF];
        lo[0] = ql[0];
        hi[0] = qh[0];
        lo[1] = ml[0];
        hi[1] = mh[0];
        lo[2] = __dadd_rd(__dadd_rd(__dmul_rd(h2, ql[0]), ql[1]), ql[2]);
        hi[2] = __dadd_ru(__dadd_ru(__dmul_ru(h2, qh[0]), qh[1]), qh[2]);
        lo[3] = __dadd_rd(__dadd_rd(__dmul_rd(h, __dsqrt_rd(ql[0])), __dsqrt_rd(ql[1])), __dsqrt_rd(ql[2]));
        hi[3] = __dadd_ru(__dadd_ru(__dmul_ru(h, __dsqrt_ru(qh[0])), __dsqrt_ru(qh[1])), __dsqrt_ru(qh[2]));
        lo[4] = fmax(ml[0], fmax(__dmul_rd(g, ml[1]), __dmul_rd(g, ml[2])));
        hi[4] = fmax(mh[0], fmax(__dmul_ru(g, mh[1]), __dmul_ru(g, mh[2])));
        lo[5] = __dadd_rd(__dadd_rd(ml[0], __dmul_rd(g, ml[1])), __dmul_rd(g, ml[2]));
        hi[5] = __dadd_ru(__dadd_ru(mh[0], __dmul_ru(g, mh[1])), __dmul_ru(g, mh[2]));
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (w.mask & (1 << f)) {
                w.vlo[f * np + q] = lo[f];
                w.vhi[f * np + q] = hi[f];
                lb[f] = lo[f];
                ub[f] = hi[f];
            }
        }
        w.flag[q] = 0;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        double v = lb[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0 && (w.mask & (1 << f))) atomic_max_nonneg(&w.scal[2 + f], v);
        if (w.law >= 1) {
            double u = ub[f];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u = fmin(u, __shfl_xor_sync(0xffffffffu, u, o));
            if ((threadIdx.x & 31) == 0 && (w.mask & (1 << f))) atomic_min_nonneg(&w.scal[16 + f], u);
        }
    }
}

// pairs whose interval may hold a feature's maximum (linear law: or its
// minimum, lo <= the smallest upper bound) go to the exact queue
__global__ void candidates_kernel(McilWork w) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= w.np) return;
    bool cand = false;
#pragma unroll
    for (int f = 0; f < NF; ++f)
        if (w.mask & (1 << f)) {
            cand |= w.vhi[f * w.np + q] >= __longlong_as_double((long long)w.scal[2 + f]);
            if (w.law >= 1) cand |= w.vlo[f * w.np + q] <= read_min_nonneg(&w.scal[16 + f]);
        }
    if (cand) {
        w.flag[q] = 1;
        const unsigned long long slot = atomicAdd(&w.scal[0], 1ull);
        w.queue[slot] = q;
    }
}

// ---------------------------------------------------------------------------
// 4. exact evaluation: one CTA (256 threads) per queued pair
// ---------------------------------------------------------------------------
struct Arr3 {
    const float *a1[3], *a2[3];
    int64_t ld1[3], ld2[3], d[3];
};

// the six features of pair q from its exact squared distances qv and
// maxima mv of the three arrays, each one FP64 expression rounded to nearest
__device__ void exact_store(McilWork &w, int64_t q, const double (&qv)[3], const double (&mv)[3], double h,
                            double h2, double g) {
    const int64_t np = w.np;
    double v[NF];
    v[0] = qv[0];
    v[1] = mv[0];
    v[2] = __dadd_rn(__dadd_rn(__dmul_rn(h2, qv[0]), qv[1]), qv[2]);
    v[3] = __dadd_rn(__dadd_rn(__dmul_rn(h, __dsqrt_rn(qv[0])), __dsqrt_rn(qv[1])), __dsqrt_rn(qv[2]));
    {
        const double bx = __dmul_rn(g, mv[1]), by = __dmul_rn(g, mv[2]);
        const double b = bx > by ? bx : by;
        v[4] = mv[0] > b ? mv[0] : b;
    }
    v[5] = __dadd_rn(__dadd_rn(mv[0], __dmul_rn(g, mv[1])), __dmul_rn(g, mv[2]));
    for (int f = 0; f < NF; ++f)
        if (w.mask & (1 << f)) w.vex[f * np + q] = v[f];
    w.flag[q] = 2;
    atomicAdd(&w.scal[10], 1ull);
}

// queued pairs from scal[start_slot] (0: from the start) to the end, one
// CTA per pair taking its arrays in turn (queues longer than EX_CAP;
// exact_split_kernel takes the rest)
__global__ void __launch_bounds__(256) exact_kernel(McilWork w, Arr3 A, double h, double h2, double g,
                                                    int start_slot) {
    __shared__ XdShared<256> sh;
    const unsigned long long nq = w.scal[0];
    const unsigned long long first = start_slot == 0 ? 0ull : w.scal[start_slot];
    if (nq <= first + (unsigned long long)EX_CAP) return;
    const int na = (w.mask & 0x3C) != 0 ? 3 : 1;
    for (unsigned long long e = first + blockIdx.x; e < nq; e += gridDim.x) {
        const int64_t q = w.queue[e];
        const int64_t i = q / w.n2, j = q - i * w.n2;
        double qv[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
        for (int a = 0; a < na; ++a) {
            double m = 0.0;
            const double v = xd_block<256, true>(A.a1[a] + i * A.ld1[a], A.a2[a] + j * A.ld2[a], A.d[a], sh, &m);
            qv[a] = v;
            mv[a] = m;
        }
        if (threadIdx.x == 0) exact_store(w, q, qv, mv, h, h2, g);
        __syncthreads();
    }
}

// The same exact evaluation spread over CTAs: one CTA per (queued pair,
// pattern array); the last CTA of a pair to finish forms its features.
// Takes the queue from scal[start_slot] when it holds at most EX_CAP pairs
// (exact_kernel takes longer queues); arrive[] cleared by the caller.
__global__ void __launch_bounds__(256) exact_split_kernel(McilWork w, Arr3 A, double h, double h2, double g,
                                                          int start_slot) {
    __shared__ XdShared<256> sh;
    const unsigned long long nq = w.scal[0], first = start_slot == 0 ? 0ull : w.scal[start_slot];
    const unsigned long long cnt = nq > first ? nq - first : 0ull;
    if (cnt > (unsigned long long)EX_CAP) return;
    const int na = (w.mask & 0x3C) != 0 ? 3 : 1;
    const unsigned long long items = cnt * (unsigned long long)na;
    for (unsigned long long it = blockIdx.x; it < items; it += gridDim.x) {
        const unsigned long long sl = it / (unsigned long long)na;
        const int a = (int)(it - sl * (unsigned long long)na);
        const int64_t q = w.queue[first + sl];
        const int64_t i = q / w.n2, j = q - i * w.n2;
        double m = 0.0;
        const double v = xd_block<256, true>(A.a1[a] + i * A.ld1[a], A.a2[a] + j * A.ld2[a], A.d[a], sh, &m);
        if (threadIdx.x == 0) {
            double *gp = w.grp + (sl * 3 + a) * 2;
            gp[0] = v;
            gp[1] = m;
            __threadfence();
            if (atomicAdd(&w.arrive[sl], 1u) == (unsigned)(na - 1)) {
                __threadfence();
                double qv[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
                for (int a2 = 0; a2 < na; ++a2) {
                    const volatile double *gq = w.grp + (sl * 3 + a2) * 2;
                    qv[a2] = gq[0];
                    mv[a2] = gq[1];
                }
                exact_store(w, q, qv, mv, h, h2, g);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 4b. tier 2 for the pairs classification left open: per pattern array, the
//     squared distance from FP32 error-free transformations (s = fl(x - y)
//     and e with s + e = x - y exactly; s^2 = p + pe exactly; 2 s e rounded;
//     e^2 dropped; per thread an error-free (H, L) accumulation), as an
//     interval that holds the exact sum (the bound of the single-norm
//     tier 2), and the maximum of |x - y| without FP64 work per
//     element: |x - y| = |s| + sign(s) e orders like the pair
//     (|s|, sign(s) e), compared lexicographically in FP32; the winner's
//     |s| + sign(s) e rounded to FP64 is the defined value (FP64 rounding
//     is monotone, so it is the maximum of the rounded differences).
// ---------------------------------------------------------------------------
struct MaxKey {
    float a, b;   // |s|, sign(s) e
};
__device__ __forceinline__ MaxKey mk_max(MaxKey u, MaxKey v) {
    return (v.a > u.a || (v.a == u.a && v.b > u.b)) ? v : u;
}

__device__ void t2_q_m(const float *x, const float *y, int64_t d, double *sred, double &qlo, double &qhi,
                       double &m) {
    float H = 0.f, L = 0.f;
    MaxKey key{0.f, 0.f};
    for (int64_t t = threadIdx.x; t < d; t += 256) {
        const float a = __ldg(x + t), bv = __ldg(y + t);
        const float sd = a - bv;
        const float bb = sd - a;
        const float e = (a - (sd - bb)) + (-bv - bb);
        const float p = sd * sd;
        const float pe = fmaf(sd, sd, -p);
        const float cr = (2.f * sd) * e;
        const float sH = H + p;                  // H += p without error, into (H, L)
        const float b2 = sH - H;
        L += (H - (sH - b2)) + (p - b2);
        H = sH;
        L += pe + cr;
        const MaxKey k{fabsf(sd), sd < 0.f ? -e : e};
        key = mk_max(key, k);
    }
    double v = (double)H + (double)L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        const MaxKey k{__shfl_xor_sync(0xffffffffu, key.a, o), __shfl_xor_sync(0xffffffffu, key.b, o)};
        key = mk_max(key, k);
    }
    __syncthreads();
    if (lane == 0) {
        sred[warp] = v;
        sred[8 + warp] = (double)key.a + (double)key.b;   // |x - y| of that element, rounded to FP64
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double D2 = 0.0, mm = 0.0;
        for (int gi = 0; gi < 8; ++gi) {
            D2 += sred[gi];
            mm = fmax(mm, sred[8 + gi]);
        }
        const double n = (double)((d + 255) / 256);
        const double rel = 2.0 * (2.9e-14 + 2.0 * n * (n + 4.0) * 3.56e-15 + 300.0 * 1.12e-16);
        const double err = rel * fabs(D2) + 1e-300;
        sred[16] = fmax(D2 - err, 0.0);
        sred[17] = D2 + err;
        sred[18] = mm;
    }
    __syncthreads();
    qlo = sred[16];
    qhi = sred[17];
    m = sred[18];
}

// queued pairs from scal[start_slot] (0: from the start) to the end
__global__ void __launch_bounds__(256) tier2_kernel_m(McilWork w, Arr3 A, double h, double h2, double g,
                                                      int start_slot) {
    __shared__ double sred[19];
    const unsigned long long nq = w.scal[0], first = start_slot == 0 ? 0ull : w.scal[start_slot];
    const bool deriv = (w.mask & 0x3C) != 0;
    for (unsigned long long e = first + blockIdx.x; e < nq; e += gridDim.x) {
        const int64_t q = w.queue[e];
        const int64_t i = q / w.n2, j = q - i * w.n2;
        double ql[3] = {0, 0, 0}, qh[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            if (a == 0 || deriv) t2_q_m(A.a1[a] + i * A.ld1[a], A.a2[a] + j * A.ld2[a], A.d[a], sred, ql[a], qh[a], mv[a]);
        if (threadIdx.x == 0) {
            const int64_t np = w.np;
            double lo[NF], hi[NF];
            lo[0] = ql[0];
            hi[0] = qh[0];
            lo[1] = hi[1] = mv[0];
            lo[2] = __dadd_rd(__dadd_rd(__dmul_rd(h2, ql[0]), ql[1]), ql[2]);
            hi[2] = __dadd_ru(__dadd_ru(__dmul_ru(h2, qh[0]), qh[1]), qh[2]);
            lo[3] = __dadd_rd(__dadd_rd(__dmul_rd(h, __dsqrt_rd(ql[0])), __dsqrt_rd(ql[1])), __dsqrt_rd(ql[2]));
            hi[3] = __dadd_ru(__dadd_ru(__dmul_ru(h, __dsqrt_ru(qh[0])), __dsqrt_ru(qh[1])), __dsqrt_ru(qh[2]));
            // the maxima are exact: the max features are evaluated exactly as
            // in the defining expression
            {
                const double bx = __dmul_rn(g, mv[1]), by = __dmul_rn(g, mv[2]);
                const double b = bx > by ? bx : by;
                lo[4] = hi[4] = mv[0] > b ? mv[0] : b;
            }
            lo[5] = hi[5] = __dadd_rn(__dadd_rn(mv[0], __dmul_rn(g, mv[1])), __dmul_rn(g, mv[2]));
            for (int f = 0; f < NF; ++f)
                if (w.mask & (1 << f)) {
                    w.vlo[f * np + q] = lo[f];
                    w.vhi[f * np + q] = hi[f];
                }
            w.flag[q] = 3;
        }
        __syncthreads();
    }
}

__global__ void mark_kernel_m(McilWork w, int slot) {
    if (threadIdx.x == 0) w.scal[slot] = w.scal[0];
}

// after tier 2 on the candidates: raise each feature's largest lower bound
// (linear law: lower its smallest upper bound) with their tighter intervals
__global__ void lb2_kernel_m(McilWork w) {
    const unsigned long long nA = w.scal[9];
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < nA;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const int64_t q = w.queue[e];
        for (int f = 0; f < NF; ++f)
            if (w.mask & (1 << f)) {
                atomic_max_nonneg(&w.scal[2 + f], w.vlo[f * w.np + q]);
                if (w.law >= 1) atomic_min_nonneg(&w.scal[16 + f], w.vhi[f * w.np + q]);
            }
    }
}

// candidates whose interval of some feature is not a single value and may
// still hold that feature's maximum (or, linear law, its minimum) are
// evaluated exactly
__global__ void cand2_kernel_m(McilWork w) {
    const unsigned long long nA = w.scal[9];
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < nA;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const int64_t q = w.queue[e];
        bool need = false;
        for (int f = 0; f < NF; ++f) {
            if (!(w.mask & (1 << f))) continue;
            const double lo = w.vlo[f * w.np + q], hi = w.vhi[f * w.np + q];
            need |= (lo < hi) && hi >= __longlong_as_double((long long)w.scal[2 + f]);
            if (w.law >= 1) need |= (lo < hi) && lo <= read_min_nonneg(&w.scal[16 + f]);
        }
        if (need) {
            w.flag[q] = 1;
            const unsigned long long slot = atomicAdd(&w.scal[0], 1ull);
            w.queue[slot] = q;
        }
    }
}

// ---------------------------------------------------------------------------
// 5. radii from the exact maxima; thresholds
// ---------------------------------------------------------------------------
// the fitted decay of the power law (the same definition as the
// single-feature correlation integral's): the smallest double whose M-th
// power, M - 1 sequential products rounded to nearest, reaches c, by
// halving [1, c]; 1 when c <= 1, +inf when c is not finite
__device__ double fitted_b_m(double c, int M) {
    if (!(c < __longlong_as_double(0x7ff0000000000000ll))) return __longlong_as_double(0x7ff0000000000000ll);
    if (!(c > 1.0)) return 1.0;
    double lo = 1.0, hi = c;
    for (int it = 0; it < 400; ++it) {
        const double half = __dmul_rn(__dsub_rn(hi, lo), 0.5);
        const double mid = __dadd_rn(lo, half);
        if (!(mid > lo) || !(mid < hi)) break;
        double pw = mid;
        for (int k = 1; k < M; ++k) pw = __dmul_rn(pw, mid);
        if (pw < c) lo = mid;
        else hi = mid;
    }
    return hi;
}

__global__ void radii_kernel_m(McilWork w, double b, const double *__restrict__ radii_in, double *radii_out) {
    // one warp per feature; the maximum is among the queued candidates
    const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long nq = w.scal[0], nA = w.scal[9];
    if (threadIdx.x == 0) w.scal[1] = nq;   // end of the candidate phase
    if (f >= NF || !(w.mask & (1 << f))) return;
    if (w.law == 3) {   // given radii [K][M+1] (R0 first, copied, not used)
        if (lane != 0) return;
        int slot = 0;
        for (int f2 = 0; f2 < f; ++f2) slot += (w.mask >> f2) & 1;
        const double *Ri = radii_in + (int64_t)slot * (w.M + 1);
        double *R = radii_out + (int64_t)slot * (w.M + 1);
        R[0] = Ri[0];
        for (int k = 1; k <= w.M; ++k) {
            const double r = Ri[k];
            R[k] = r;
            w.thr[f * 32 + k - 1] = feat_squared(f) ? __dmul_rn(r, r) : r;
        }
        return;
    }
    // every pair that may hold the maximum (or the minimum) now has its
    // value exactly: from the exact pass (flag 2) or a single-value
    // tier-2 interval; every other candidate's value lies strictly inside
    // (smallest upper bound, largest lower bound)
    double mx = 0.0, mn = __longlong_as_double(0x7ff0000000000000ll);
    for (unsigned long long e = lane; e < nA; e += 32) {
        const int64_t q = w.queue[e];
        const double lo = w.vlo[f * w.np + q], hi = w.vhi[f * w.np + q];
        double v = -1.0;
        if (w.flag[q] == 2) v = w.vex[f * w.np + q];
        else if (lo == hi) v = lo;
        if (v >= 0.0) {
            mx = fmax(mx, v);
            mn = fmin(mn, v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (lane == 0) {
        int slot = 0;
        for (int f2 = 0; f2 < f; ++f2) slot += (w.mask >> f2) & 1;
        double *R = radii_out + (int64_t)slot * (w.M + 1);
        double r = feat_squared(f) ? __dsqrt_rn(mx) : mx;
        R[0] = r;
        const double R0 = r;
        const double Rm = feat_squared(f) ? __dsqrt_rn(mn) : mn;
        const double hl = w.law == 1 ? __ddiv_rn(__dsub_rn(R0, Rm), (double)w.M) : 0.0;
        const double bf = w.law == 2 ? fitted_b_m(__ddiv_rn(R0, Rm), w.M) : b;
        for (int k = 1; k <= w.M; ++k) {
            r = w.law == 1 ? __dsub_rn(R0, __dmul_rn((double)k, hl)) : __ddiv_rn(r, bf);
            R[k] = r;
            w.thr[f * 32 + k - 1] = feat_squared(f) ? __dmul_rn(r, r) : r;
        }
    }
}

// ---------------------------------------------------------------------------
// 6. classify by interval; undecided pairs join the exact queue
// ---------------------------------------------------------------------------
// first = 0: pairs still on their tier-1 interval (flag 0); first = 1:
// pairs tier 2 re-bounded (flag 3).  Undecided ones join the queue.
__global__ void classify_kernel_m(McilWork w, int second) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= w.np || w.flag[q] != (second ? 3 : 0)) return;
    bool undecided = false;
    for (int f = 0; f < NF && !undecided; ++f) {
        if (!(w.mask & (1 << f))) continue;
        const double lo = w.vlo[f * w.np + q], hi = w.vhi[f * w.np + q];
        for (int k = 0; k < w.M; ++k) {
            const double T = w.thr[f * 32 + k];
            if (!(hi < T) && !(lo >= T)) { undecided = true; break; }
        }
    }
    if (undecided) {
        w.flag[q] = 1;
        const unsigned long long slot = atomicAdd(&w.scal[0], 1ull);
        w.queue[slot] = q;
    }
}

// ---------------------------------------------------------------------------
// 7. bins (exact value where evaluated, else the interval) and counts
// ---------------------------------------------------------------------------
__global__ void bins_kernel_m(McilWork w, uint8_t *__restrict__ bins, int64_t *__restrict__ counts) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int slot = 0;
    for (int f = 0; f < NF; ++f) {
        if (!(w.mask & (1 << f))) continue;
        int K = 0;
        if (q < w.np) {
            const bool ex = w.flag[q] == 2;
            const double v = ex ? w.vex[f * w.np + q] : w.vhi[f * w.np + q];
            for (int k = 0; k < w.M; ++k)
                if (v < w.thr[f * 32 + k]) K = k + 1;
            bins[(int64_t)slot * w.np + q] = (uint8_t)K;
        }
        for (int k = 0; k < w.M; ++k) {
            const unsigned c = __popc(__ballot_sync(0xffffffffu, K > k));
            if (lane == 0 && c) atomicAdd((unsigned long long *)&counts[(int64_t)slot * w.M + k], (unsigned long long)c);
        }
        ++slot;
    }
}

__global__ void finish_kernel_m(McilWork w, const unsigned long long *t0, const unsigned long long *t1,
                                const unsigned long long *t2, int64_t *counts, double *Cv, int K,
                                int64_t *n_exact) {
    const bool to = (t0 && *t0) || (t1 && *t1) || (t2 && *t2);
    if (threadIdx.x == 0 && n_exact) *n_exact = to ? -2 : (int64_t)w.scal[10];
    if (Cv)
        for (int e = threadIdx.x; e < K * w.M; e += blockDim.x)
            Cv[e] = __ddiv_rn((double)counts[e], (double)w.np);
}

static rd_status mcil_check(int64_t n1, int64_t n2, int Gy, int Gx, int nsp, int mask, int M, double b) {
    if (n1 < 1 || n2 < 1 || n1 > 65535 || n2 > 65535) return RD_ERR_INVALID_ARG;
    if (Gx < 2 || Gx > 4096 || Gy < 1 || Gy > 4096 || nsp < 1 || nsp > 2) return RD_ERR_INVALID_ARG;
    if ((int64_t)nsp * Gy * Gx > XD_MAX_D) return RD_ERR_INVALID_ARG;
    if (mask < 1 || mask > 63 || M < 1 || M > 32 || !(b > 1.0)) return RD_ERR_INVALID_ARG;
    return RD_OK;
}

}  // namespace rdcil

using namespace rdcil;

static rd_status mcil_run(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2, int64_t n2,
                          int32_t Gy, int32_t Gx, int32_t n_species, int32_t features, int32_t scale, double b,
                          int law, int32_t M, double *d_radii_out, uint8_t *d_bins, int64_t *d_counts, double *d_C,
                          int64_t *d_n_exact, void *d_work, size_t work_bytes, void *stream,
                          const double *d_radii_in = nullptr) {
    if (law == 3 && !d_radii_in) return RD_ERR_INVALID_ARG;
    rd_status st = mcil_check(n1, n2, Gy, Gx, n_species, features, M, b);
    if (st) return st;
    const int64_t d0 = (int64_t)n_species * Gy * Gx;
    if (!d_X1 || !d_X2 || !d_radii_out || !d_bins || !d_counts || !d_work) return RD_ERR_INVALID_ARG;
    if (ld1 < d0 || ld2 < d0 || (((uintptr_t)d_work) & 255)) return RD_ERR_INVALID_ARG;
    McilWork w = mlayout(n1, n2, Gy, Gx, n_species, features, scale, M, d_work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    w.law = law;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = __builtin_popcount((unsigned)features);
    const int64_t np = w.np;
    const unsigned gp = (unsigned)((np + 255) / 256);
    RD_CUDA_TRY(cudaMemsetAsync(w.scal, 0, MC_SCAL * sizeof(unsigned long long), s));
    RD_CUDA_TRY(cudaMemsetAsync(d_counts, 0, (size_t)K * M * sizeof(int64_t), s));

    // patterns (scaled copies when asked)
    const float *P1 = d_X1, *P2 = d_X2;
    int64_t l1 = ld1, l2 = ld2;
    if (scale) {
        minmax_kernel<<<(unsigned)(n1 * n_species), 256, 0, s>>>(d_X1, ld1, (int64_t)Gy * Gx, n_species, w.S1);
        note_launch();
        minmax_kernel<<<(unsigned)(n2 * n_species), 256, 0, s>>>(d_X2, ld2, (int64_t)Gy * Gx, n_species, w.S2);
        note_launch();
        P1 = w.S1; P2 = w.S2; l1 = l2 = d0;
    }
    const bool deriv = (features & 0x3C) != 0;
    if (deriv) {
        const int64_t r1 = n1 * n_species * Gy, r2 = n2 * n_species * Gy;
        // float4 rows need 16-byte aligned rows: Gx % 4 == 0 and pattern
        // strides and bases on 16-byte boundaries
        const bool vec = (Gx % 4 == 0) && (l1 % 4 == 0) && (l2 % 4 == 0) && ((((uintptr_t)P1) | ((uintptr_t)P2)) % 16 == 0);
        if (vec) {
            const int64_t b1 = (r1 + 7) / 8, b2 = (r2 + 7) / 8;
            fd4_kernel<<<(unsigned)(b1 < 65535 * 16 ? b1 : 65535 * 16), 256, 0, s>>>(P1, l1, n1, Gy, Gx, n_species,
                                                                                    w.Ax1, w.Ay1);
            note_launch();
            fd4_kernel<<<(unsigned)(b2 < 65535 * 16 ? b2 : 65535 * 16), 256, 0, s>>>(P2, l2, n2, Gy, Gx, n_species,
                                                                                    w.Ax2, w.Ay2);
        } else {
            // one block per grid row (every row's loads in flight at once)
            const int fdt = Gx >= 256 ? 256 : (Gx >= 128 ? 128 : 64);
            fd_kernel<<<(unsigned)(r1 < 0x7FFFFFFF ? r1 : 0x7FFFFFFF), fdt, 0, s>>>(P1, l1, n1, Gy, Gx, n_species,
                                                                                   w.Ax1, w.Ay1);
            note_launch();
            fd_kernel<<<(unsigned)(r2 < 0x7FFFFFFF ? r2 : 0x7FFFFFFF), fdt, 0, s>>>(P2, l2, n2, Gy, Gx, n_species,
                                                                                   w.Ax2, w.Ay2);
        }
        note_launch();
    }
    Arr3 A{};
    A.a1[0] = P1; A.a2[0] = P2; A.ld1[0] = l1; A.ld2[0] = l2; A.d[0] = d0;
    A.a1[1] = w.Ax1; A.a2[1] = w.Ax2; A.a1[2] = w.Ay1; A.a2[2] = w.Ay2;
    A.ld1[1] = A.ld2[1] = A.d[1] = w.dex;
    A.ld1[2] = A.ld2[2] = A.d[2] = w.dey;

    // squared distances: tier-1 intervals
    QIv qi{};
    const unsigned long long *tmo[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < 3; ++a) {
        if (!w.cw[a]) continue;
        st = cil_tier1_intervals(A.a1[a], A.ld1[a], n1, A.a2[a], A.ld2[a], n2, A.d[a], w.cw[a], w.cw_bytes[a],
                                 &qi.lo[a], &qi.hi[a], &tmo[a], s);
        if (st) return st;
    }
    // maxima
    RD_CUDA_TRY(cudaMemsetAsync(w.mabs, 0, sizeof(float) * 3 * np, s));
    const bool need_m0 = (features & 0x32) != 0, need_md = (features & 0x30) != 0;
    for (int a = 0; a < 3; ++a) {
        if ((a == 0 ? !need_m0 : !need_md) || A.d[a] == 0) continue;
        // tile shape: 64 x 256 pairs when set 1 is small (less padding),
        // else 128 x 128; K chunks (multiples of 32, at least 64) for about
        // two CTAs per SM
        const bool narrow = n1 <= 64;
        const int64_t TA = narrow ? 64 : 128, TB = narrow ? 256 : 128;
        const int64_t tiles = ((n1 + TA - 1) / TA) * ((n2 + TB - 1) / TB);
        const int64_t want = (2 * 148 + tiles - 1) / tiles;
        int64_t kch = (A.d[a] + want - 1) / want;
        kch = (kch + MX_K - 1) / MX_K * MX_K;
        if (kch < 2 * MX_K) kch = 2 * MX_K;
        const int64_t nk = (A.d[a] + kch - 1) / kch;
        dim3 grid((unsigned)((n2 + TB - 1) / TB), (unsigned)((n1 + TA - 1) / TA), (unsigned)nk);
        if (narrow) {
            // the attribute belongs to the current device: set it on every call
            RD_CUDA_TRY(cudaFuncSetAttribute(maxabs_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)MaxTile<64>::SMEM));
            maxabs_kernel<64><<<grid, 256, MaxTile<64>::SMEM, s>>>(A.a1[a], A.ld1[a], n1, A.a2[a], A.ld2[a], n2,
                                                                   A.d[a], kch, w.mabs + a * np);
        } else {
            RD_CUDA_TRY(cudaFuncSetAttribute(maxabs_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)MaxTile<128>::SMEM));
            maxabs_kernel<128><<<grid, 256, MaxTile<128>::SMEM, s>>>(A.a1[a], A.ld1[a], n1, A.a2[a], A.ld2[a], n2,
                                                                     A.d[a], kch, w.mabs + a * np);
        }
        note_launch();
    }
    const double g = (double)(Gx - 1), h = 1.0 / g, h2 = 1.0 / (g * g);
    intervals_kernel<<<gp, 256, 0, s>>>(w, qi, h, h2, g);
    note_launch();
    if (law != 3) {   // given radii need no maxima or minima
        candidates_kernel<<<gp, 256, 0, s>>>(w);
        note_launch();
    }
    mark_kernel_m<<<1, 32, 0, s>>>(w, 9);
    note_launch();
    const unsigned ge = 4 * 148;
    tier2_kernel_m<<<ge, 256, 0, s>>>(w, A, h, h2, g, 0);
    note_launch();
    lb2_kernel_m<<<148, 256, 0, s>>>(w);
    note_launch();
    cand2_kernel_m<<<148, 256, 0, s>>>(w);
    note_launch();
    RD_CUDA_TRY(cudaMemsetAsync(w.arrive, 0, sizeof(unsigned int) * EX_CAP, s));
    exact_split_kernel<<<2 * 148, 256, 0, s>>>(w, A, h, h2, g, 9);
    note_launch();
    exact_kernel<<<ge, 256, 0, s>>>(w, A, h, h2, g, 9);
    note_launch();
    radii_kernel_m<<<1, 32 * NF, 0, s>>>(w, b, d_radii_in, d_radii_out);
    note_launch();
    classify_kernel_m<<<gp, 256, 0, s>>>(w, 0);
    note_launch();
    tier2_kernel_m<<<ge, 256, 0, s>>>(w, A, h, h2, g, 1);
    note_launch();
    mark_kernel_m<<<1, 32, 0, s>>>(w, 8);
    note_launch();
    classify_kernel_m<<<gp, 256, 0, s>>>(w, 1);
    note_launch();
    RD_CUDA_TRY(cudaMemsetAsync(w.arrive, 0, sizeof(unsigned int) * EX_CAP, s));
    exact_split_kernel<<<2 * 148, 256, 0, s>>>(w, A, h, h2, g, 8);
    note_launch();
    exact_kernel<<<ge, 256, 0, s>>>(w, A, h, h2, g, 8);
    note_launch();
    bins_kernel_m<<<gp, 256, 0, s>>>(w, d_bins, d_counts);
    note_launch();
    finish_kernel_m<<<1, 256, 0, s>>>(w, tmo[0], tmo[1], tmo[2], d_counts, d_C, K, d_n_exact);
    note_launch();
    return cuda_status(cudaGetLastError());
}

extern "C" rd_status mcil_workspace_size(int64_t n1, int64_t n2, int32_t G, int32_t n_species, int32_t features,
                                         int32_t scale, int32_t M, size_t *bytes) {
    return mcil_workspace_size_rect(n1, n2, G, G, n_species, features, scale, M, bytes);
}

extern "C" rd_status mcil_workspace_size_rect(int64_t n1, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                              int32_t features, int32_t scale, int32_t M, size_t *bytes) {
    if (!bytes) return RD_ERR_INVALID_ARG;
    rd_status st = mcil_check(n1, n2, Gy, Gx, n_species, features, M, 2.0);
    if (st) return st;
    *bytes = mlayout(n1, n2, Gy, Gx, n_species, features, scale, M, nullptr).bytes;
    return RD_OK;
}

extern "C" rd_status mcil_features(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2,
                                   int64_t n2, int32_t G, int32_t n_species, int32_t features, int32_t scale,
                                   double b, int32_t M, double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                                   double *d_C, int64_t *d_n_exact, void *d_work, size_t work_bytes, void *stream) {
    return mcil_run(d_X1, ld1, n1, d_X2, ld2, n2, G, G, n_species, features, scale, b, 0, M, d_radii_out, d_bins,
                    d_counts, d_C, d_n_exact, d_work, work_bytes, stream);
}

extern "C" rd_status mcil_features_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2,
                                        int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species, int32_t features,
                                        int32_t scale, double b, int32_t M, double *d_radii_out, uint8_t *d_bins,
                                        int64_t *d_counts, double *d_C, int64_t *d_n_exact, void *d_work,
                                        size_t work_bytes, void *stream) {
    return mcil_run(d_X1, ld1, n1, d_X2, ld2, n2, Gy, Gx, n_species, features, scale, b, 0, M, d_radii_out, d_bins,
                    d_counts, d_C, d_n_exact, d_work, work_bytes, stream);
}

extern "C" rd_status mcil_features_fitted_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                               int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                               int32_t features, int32_t scale, int32_t M, double *d_radii_out,
                                               uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_exact,
                                               void *d_work, size_t work_bytes, void *stream) {
    return mcil_run(d_X1, ld1, n1, d_X2, ld2, n2, Gy, Gx, n_species, features, scale, 2.0, 2, M, d_radii_out,
                    d_bins, d_counts, d_C, d_n_exact, d_work, work_bytes, stream);
}

extern "C" rd_status mcil_features_linear_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                               int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                               int32_t features, int32_t scale, int32_t M, double *d_radii_out,
                                               uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_exact,
                                               void *d_work, size_t work_bytes, void *stream) {
    return mcil_run(d_X1, ld1, n1, d_X2, ld2, n2, Gy, Gx, n_species, features, scale, 2.0, 1, M, d_radii_out,
                    d_bins, d_counts, d_C, d_n_exact, d_work, work_bytes, stream);
}

extern "C" rd_status mcil_features_given_rect(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                              int64_t ld2, int64_t n2, int32_t Gy, int32_t Gx, int32_t n_species,
                                              int32_t features, int32_t scale, int32_t M,
                                              const double *d_radii_in, double *d_radii_out, uint8_t *d_bins,
                                              int64_t *d_counts, double *d_C, int64_t *d_n_exact, void *d_work,
                                              size_t work_bytes, void *stream) {
    return mcil_run(d_X1, ld1, n1, d_X2, ld2, n2, Gy, Gx, n_species, features, scale, 2.0, 3, M, d_radii_out, d_bins,
                    d_counts, d_C, d_n_exact, d_work, work_bytes, stream, d_radii_in);
}
