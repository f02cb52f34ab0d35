// Correlation integral of two pattern sets (eq. eCDF, eq. CIL, Sec. 2.1).
//
// Exactness contract.  For every pair the library decides K_ij =
// #{k : d2_ij < R_k^2} for d2_ij = the real number sum_t (x_t - y_t)^2 of
// the FP32 inputs rounded once to the nearest double (the distance of
// Sec. 2.1 is defined on the reals; this value depends on no evaluation
// order).  Every bound below encloses the exact real sum S; since rounding
// to nearest is monotone, an interval with representable ends that holds S
// also holds d2 = fl64(S).  It does so in three stages:
//   1. pack:  centre every pattern by c = the mean of up to 16 patterns
//      sampled from each set (translation does not change distances; any c
//      is valid, a central one keeps the bf16 split accurate), split x - c
//      into bf16 hi + lo, and record per
//      pattern N = |hi+lo|^2, H = |hi| + |lo|, L = |lo| and the
//      representation error E = |(x - c) - (hi + lo)| (all FP64);
//   2. Gram:  P_ij = hi_i.hi_j + hi_i.lo_j + lo_i.hi_j (three bf16
//      products, the default), or P_ij = hi_i.hi_j alone when asked (one
//      product: a third of the tensor-core work and half its operand bytes,
//      for a wider interval); FP32 accumulation per K chunk in tensor
//      memory, chunk partials summed with TwoSum into FP32 hi/lo pairs per
//      K segment, segments combined the same way;
//   3. tier 1: A = N_i + N_j - 2 P_ij approximates d2_ij with a rigorous
//      error bound (FP32 accumulation model, the dropped terms: lo.lo, and
//      for one product hi.lo + lo.hi, each by Cauchy-Schwarz on the parts'
//      norms; E_i + E_j), kept as an FP32 interval rounded outwards;
//   4. tier 2: pairs whose interval could hold the maximum (which defines R0)
//      or contain a threshold get an FP32 error-free evaluation of the exact
//      sum of squares (TwoSum / exact products, double-float accumulation)
//      with a ~1e-12 relative bound;
//   5. tier 3: the few pairs still undecided (in practice the maximum) are
//      evaluated exactly (integer fixed-point accumulation, one rounding;
//      exact.cuh), one CTA per pair.
// Counts per radius are reduced with warp ballot + popc.
#include <atomic>
#include <cstdio>
#include <cuda_bf16.h>
#include "common.cuh"
#include "exact.cuh"

namespace rdcil {

rd_status launch_gram_tc(const void *hi, const void *lo, int64_t n1, int64_t n2, int64_t dp, int64_t S,
                         int64_t cs, int np_, float *Ppart, uint32_t *status, cudaStream_t s);

// longest accumulator chunk, in K steps of 64 (bounds the FP32 accumulation
// error), for three products / one product: with one product the dropped
// cross terms dominate the bound, so longer chunks (fewer drains) cost
// nothing in interval width
static constexpr int KSTEPS_MAX = 4, KSTEPS_MAX1 = 16;
static constexpr int PAD = 64;           // padded pattern length granularity
static constexpr int TILE = 128;         // Gram output tile (pairs per side)
// tier 3: queues of at most EXS_CAP pairs are spread over CTAs by segments of
// EXS_SEG elements (every pair's exact digit sums meet in global memory);
// longer queues take one CTA per pair
static constexpr int EXS_CAP = 64, EXS_SEG = 2048;
static constexpr int N_SM = 148;

static inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// b^-2k, k = 1..M, evaluated on the host (only used for the threshold
// ranges, which carry a relative margin)
struct Beta {
    double v[32];
};

// scalar slots of the workspace
enum : int {
    SC_LB1 = 0,    // max over pairs of the tier-1 lower bound (float bits)
    SC_UB1 = 1,    // max over pairs of the tier-1 upper bound (float bits)
    SC_LB2 = 2,    // max over maximum candidates of the tier-2 lower bound (double bits)
    SC_UB2 = 3,    // max over maximum candidates of the tier-2 upper bound (double bits)
    SC_MAX = 4,    // exact maximum (double bits)
    SC_Q1 = 5,     // tier-2 queue length
    SC_Q2 = 6,     // tier-3 queue length
    SC_UNDECIDED = 7,
    SC_TIMEOUT = 8,
    // linear radii law: the smallest distance, kept as minima through
    // atomicMax of complemented bit patterns (the slots start at 0)
    SC_LBM1 = 9,   // min over pairs of the tier-1 lower bound
    SC_UBM1 = 10,  // min over pairs of the tier-1 upper bound
    SC_LBM2 = 11,  // min over minimum candidates of the tier-2 lower bound
    SC_UBM2 = 12,  // min over minimum candidates of the tier-2 upper bound
    SC_MIN = 13,   // exact minimum
};

// queue entries: pair index | bit 63 maximum candidate | bit 62 minimum candidate
static constexpr unsigned long long Q_MAX = 1ull << 63, Q_MIN = 1ull << 62, Q_IDX = Q_MIN - 1;

// radii laws (Sec. 2.1): R_k = R_{k-1} / b, R_k = R0 - k (R0 - R_min) / M,
// or R_k = R_{k-1} / b with b fitted so that R_M = R_min (see fitted_b)
enum : int { LAW_POWER = 0, LAW_LINEAR = 1, LAW_FITTED = 2 };
__host__ __device__ constexpr bool law_needs_min(int law) { return law == LAW_LINEAR || law == LAW_FITTED; }

// The fitted decay: the smallest double b whose M-th power, formed as M - 1
// sequential products rounded to nearest, reaches c = R0 / R_min, by halving
// [1, c] (mid = lo + (hi - lo) * 0.5, each operation rounded to nearest)
// until lo and hi are adjacent; 1 when c <= 1, +inf when c is not finite.
__device__ double fitted_b(double c, int M) {
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

// minima of non-negative values through atomicMax on complemented bits
__device__ __forceinline__ void atomic_min_f(unsigned long long *slot, float v) {
    atomicMax(slot, 0xFFFFFFFFull - (unsigned long long)__float_as_uint(v));
}
__device__ __forceinline__ float read_min_f(unsigned long long s) {
    return s ? __uint_as_float((unsigned)(0xFFFFFFFFull - s)) : __int_as_float(0x7f800000);
}
__device__ __forceinline__ void atomic_min_d(unsigned long long *slot, double v) {
    atomicMax(slot, ~(unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double read_min_d(unsigned long long s) {
    return s ? __longlong_as_double((long long)~s) : __longlong_as_double(0x7ff0000000000000ll);
}

struct CilWork {
    int64_t n1, n2, d, dp;
    int64_t ntj, S, cs;     // Gram: tiles along set 2, K segments per tile, K steps per chunk
    int64_t np_;            // Gram products: 3 (hi.hi + hi.lo + lo.hi) or 1 (hi.hi)
    int64_t nchunk;         // upper bound on the chunk partials summed per pair
    float *centre;          // [dp]
    __nv_bfloat16 *hi;      // [(n1+n2)][dp]
    __nv_bfloat16 *lo;      // [(n1+n2)][dp]
    double *N, *H, *L, *E;  // [(n1+n2)]
    float *Hf, *Lf, *Ef;    // [(n1+n2)] the same bounds as FP32, rounded up
    float *Ppart;           // [S][n1][n2] segment sums (FP32 running sums of the chunks)
    float *lo32, *hi32;     // [n1*n2] tier-1 interval of d2 (rounded outwards)
    double *lo2, *hi2;      // [n1*n2] tier-2 interval (valid where flag >= 1)
    double *ex;             // [n1*n2] exact d2 (valid where flag == 2)
    uint8_t *flag;          // [n1*n2] 0: tier 1 decides, 1: tier 2, 2: exact
    unsigned long long *q1, *q2;  // [n1*n2] tier-2 / tier-3 queues (bit 63: may hold the maximum)
    long long *xacc;        // [EXS_CAP][XD] digit sums of the split tier 3 (zeroed per call)
    unsigned *xarr;         // [2][EXS_CAP] CTAs arrived per queued pair, non-finite flags
    float *t1lo, *t1hi;     // [32] tier-1 threshold ranges (FP32, outward)
    double *t2lo, *t2hi;    // [32] tier-2 threshold ranges
    unsigned long long *scal;  // see SC_* below
    size_t bytes;
};

// Gram product count, process-wide (cil_set_gram_products): 3 by default.
// One product halves the Gram's time at the paper's scale, but its interval
// (the cross terms' Cauchy-Schwarz bound, about 2^-8 |x_i| |x_j|) leaves
// some twenty times more pairs to tier 2 near the radii, whose per-pair
// re-evaluation then costs more than the Gram saved on the workloads
// measured; it stays available for data whose distances sit far from the
// thresholds.
static std::atomic<int> g_gram_products{3};

static int gram_products_for(int64_t, int64_t) { return g_gram_products.load(); }

static CilWork layout(int64_t n1, int64_t n2, int64_t d, void *base) {
    CilWork w{};
    w.n1 = n1; w.n2 = n2; w.d = d;
    w.dp = round_up(d, PAD);
    // Gram work split: one CTA per (128 x 128 output tile, K segment), with
    // enough segments to give every SM a CTA (at most 32 for a single tile,
    // which keeps the partials of small problems small).  Accumulator
    // chunks of one K step (64 columns) while the whole product is small,
    // else of up to KSTEPS_MAX steps: the chunk length sets the FP32
    // accumulation bound, and the drain of a chunk must keep pace with the
    // tensor core.
    const int64_t nti = (n1 + TILE - 1) / TILE, ntj = (n2 + TILE - 1) / TILE, tiles = nti * ntj;
    const int64_t n64 = w.dp / PAD;
    int64_t S = tiles == 1 ? 32 : N_SM / tiles;
    if (S < 1) S = 1;
    if (S > n64) S = n64;
    const int64_t seg_max = (n64 + S - 1) / S;
    w.ntj = ntj;
    w.S = S;
    w.np_ = gram_products_for(tiles, n64);
    const int64_t kmax = w.np_ == 1 ? KSTEPS_MAX1 : KSTEPS_MAX;
    w.cs = tiles * n64 <= 4096 ? 1 : (seg_max < kmax ? seg_max : kmax);
    w.nchunk = S * ((seg_max + w.cs - 1) / w.cs);
    int64_t n = n1 + n2;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return (char *)base + o;
    };
    w.centre = (float *)take(sizeof(float) * w.dp);
    w.hi = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * n * w.dp);
    w.lo = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * n * w.dp);
    w.N = (double *)take(sizeof(double) * n);
    w.H = (double *)take(sizeof(double) * n);
    w.L = (double *)take(sizeof(double) * n);
    w.E = (double *)take(sizeof(double) * n);
    w.Hf = (float *)take(sizeof(float) * n);
    w.Lf = (float *)take(sizeof(float) * n);
    w.Ef = (float *)take(sizeof(float) * n);
    const int64_t np = n1 * n2;
    w.Ppart = (float *)take(sizeof(float) * S * np);
    w.lo32 = (float *)take(sizeof(float) * np);
    w.hi32 = (float *)take(sizeof(float) * np);
    w.lo2 = (double *)take(sizeof(double) * np);
    w.hi2 = (double *)take(sizeof(double) * np);
    w.ex = (double *)take(sizeof(double) * np);
    w.flag = (uint8_t *)take(sizeof(uint8_t) * np);
    w.q1 = (unsigned long long *)take(sizeof(unsigned long long) * np);
    w.q2 = (unsigned long long *)take(sizeof(unsigned long long) * np);
    w.xacc = (long long *)take(sizeof(long long) * EXS_CAP * XD + sizeof(unsigned) * 2 * EXS_CAP);
    w.xarr = (unsigned *)(w.xacc + EXS_CAP * XD);
    w.t1lo = (float *)take(sizeof(float) * 32);
    w.t1hi = (float *)take(sizeof(float) * 32);
    w.t2lo = (double *)take(sizeof(double) * 32);
    w.t2hi = (double *)take(sizeof(double) * 32);
    w.scal = (unsigned long long *)take(sizeof(unsigned long long) * 16);
    w.bytes = off;
    return w;
}

// FP32 error-free sum accumulation (Knuth TwoSum): (hi, lo) holds a value
// whose lo part collects the rounding errors of the hi part.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
    float s = hi + v;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += e;
}

// ---------------------------------------------------------------------------
// 1. centre and pack
// ---------------------------------------------------------------------------
__global__ void centre_kernel(const float *__restrict__ X1, int64_t ld1, int64_t n1,
                              const float *__restrict__ X2, int64_t ld2, int64_t n2, int64_t d,
                              int64_t dp, float *__restrict__ centre) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= dp) return;
    if (t >= d) { centre[t] = 0.f; return; }
    // any centre is valid (distances are translation invariant); a good one
    // keeps |x - c| small so the bf16 split loses little.  The mean of up to
    // 16 patterns evenly spread over each set is plenty for that.
    // (all samples are loaded before they are summed, so the loads overlap)
    const int64_t s1 = n1 < 16 ? n1 : 16, s2 = n2 < 16 ? n2 : 16;
    float v1[16], v2[16];
#pragma unroll
    for (int a = 0; a < 16; ++a) {
        v1[a] = a < s1 ? X1[(a * n1 / s1) * ld1 + t] : 0.f;
        v2[a] = a < s2 ? X2[(a * n2 / s2) * ld2 + t] : 0.f;
    }
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 16; ++a) s += v1[a] + v2[a];
    centre[t] = s / (float)(s1 + s2);
}

// One element of the pack: x - c split into bf16 hi + lo, with the
// compensated square sum of hi + lo and the bound sums.
struct PackAcc {
    float nh = 0.f, nl = 0.f, sH = 0.f, sL = 0.f, sE = 0.f;
};
__device__ __forceinline__ void pack_elem(float xv, float cv, __nv_bfloat16 &h, __nv_bfloat16 &l, PackAcc &A) {
    float xc = xv - cv;
    // exact rounding error of x - c (TwoSum of x and -c)
    float bb = xc - xv;
    float dc = (xv - (xc - bb)) - (cv + bb);
    h = __float2bfloat16_rn(xc);
    float hf = __bfloat162float(h);
    float r = xc - hf;                 // exact
    l = __float2bfloat16_rn(r);
    float lf = __bfloat162float(l);
    float sv = hf + lf;                // exact
    float p = sv * sv;
    float pe = fmaf(sv, sv, -p);       // exact error of the square
    two_sum_acc(A.nh, A.nl, p);
    A.nl += pe;
    A.sH = fmaf(hf, hf, A.sH);
    A.sL = fmaf(lf, lf, A.sL);
    float e = fabsf(dc) + fabsf(r - lf);   // |(x - c) - (hi + lo)|, bounded
    A.sE = fmaf(e, e, A.sE);
}

// One block per pattern; each thread takes groups of 8 elements (float4
// loads, 16-byte bf16 stores when the pattern row is 16-byte aligned).
// lo == nullptr: the lo parts are formed (for N, L and E) but not stored
// (the one-product Gram does not read them).
__global__ void pack_kernel(const float *__restrict__ X1, int64_t ld1, int64_t n1,
                            const float *__restrict__ X2, int64_t ld2, int64_t d, int64_t dp,
                            const float *__restrict__ centre, __nv_bfloat16 *__restrict__ hi,
                            __nv_bfloat16 *__restrict__ lo, double *__restrict__ Nn, double *__restrict__ Hn,
                            double *__restrict__ Ln, double *__restrict__ En, float *__restrict__ Hf,
                            float *__restrict__ Lf, float *__restrict__ Ef) {
    const int64_t i = blockIdx.x;
    const float *x = i < n1 ? X1 + i * ld1 : X2 + (i - n1) * ld2;
    const bool vec = ((uintptr_t)x & 15) == 0;
    // N = |hi + lo|^2 to ~2^-44 relative (compensated FP32); H, L, E are
    // upper bounds (plain FP32 sums, inflated below)
    PackAcc A;
    for (int64_t t0 = (int64_t)threadIdx.x * 8; t0 < dp; t0 += (int64_t)blockDim.x * 8) {
        __align__(16) __nv_bfloat16 h[8];
        __align__(16) __nv_bfloat16 l[8];
        if (vec && t0 + 8 <= d) {
            const float4 xa = *reinterpret_cast<const float4 *>(x + t0);
            const float4 xb = *reinterpret_cast<const float4 *>(x + t0 + 4);
            const float4 ca = *reinterpret_cast<const float4 *>(centre + t0);
            const float4 cb = *reinterpret_cast<const float4 *>(centre + t0 + 4);
            pack_elem(xa.x, ca.x, h[0], l[0], A);
            pack_elem(xa.y, ca.y, h[1], l[1], A);
            pack_elem(xa.z, ca.z, h[2], l[2], A);
            pack_elem(xa.w, ca.w, h[3], l[3], A);
            pack_elem(xb.x, cb.x, h[4], l[4], A);
            pack_elem(xb.y, cb.y, h[5], l[5], A);
            pack_elem(xb.z, cb.z, h[6], l[6], A);
            pack_elem(xb.w, cb.w, h[7], l[7], A);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                h[k] = l[k] = __float2bfloat16_rn(0.f);
                if (t0 + k < d) pack_elem(x[t0 + k], centre[t0 + k], h[k], l[k], A);
            }
        }
        *reinterpret_cast<uint4 *>(hi + i * dp + t0) = *reinterpret_cast<const uint4 *>(h);
        if (lo) *reinterpret_cast<uint4 *>(lo + i * dp + t0) = *reinterpret_cast<const uint4 *>(l);
    }
    float nh = A.nh, nl = A.nl, sH = A.sH, sL = A.sL, sE = A.sE;
    __shared__ float red[5][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        // combine (hi, lo) pairs error-free across lanes
        float oh = __shfl_xor_sync(0xffffffffu, nh, o), ol = __shfl_xor_sync(0xffffffffu, nl, o);
        two_sum_acc(nh, nl, oh);
        nl += ol;
        sH += __shfl_xor_sync(0xffffffffu, sH, o);
        sL += __shfl_xor_sync(0xffffffffu, sL, o);
        sE += __shfl_xor_sync(0xffffffffu, sE, o);
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = nh; red[1][warp] = nl; red[2][warp] = sH; red[3][warp] = sL; red[4][warp] = sE; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0, e = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += (double)red[0][w] + (double)red[1][w];
            b += red[2][w]; c += red[3][w]; e += red[4][w];
        }
        // FP32 sums of at most dp non-negative terms: relative error below
        // dp * 2^-23; inflate the bounds by that much (and 1e-6 more).
        double infl = 1.0 + (double)(dp + 64) * 1.2e-7 + 1e-6;
        Nn[i] = a;
        Hn[i] = (sqrt(b * infl) + sqrt(c * infl)) * (1.0 + 1e-12);
        Ln[i] = sqrt(c * infl) * (1.0 + 1e-12);
        En[i] = sqrt(e * infl) * (1.0 + 1e-12) + 1e-300;
        Hf[i] = __double2float_ru(Hn[i]);
        Lf[i] = __double2float_ru(Ln[i]);
        Ef[i] = __double2float_ru(En[i]) + 1e-30f;
    }
}

// ---------------------------------------------------------------------------
// 2. Gram product: tensor cores (gram_tc.cu), K segments of summed chunks.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// 3. tier 1: approximate d2 and a rigorous bound, as an FP32 interval
// ---------------------------------------------------------------------------
// Accumulation model for the Gram: a sequence of n roundings into one FP32
// accumulator errs by at most n * u * S, S = sum of the magnitudes of the
// products, u the unit roundoff of one accumulation step (gam = n * u is
// passed in per Gram kernel).  Here S = sum |hi||hi'| + |hi||lo'| + |lo||hi'|
// <= H_i H_j (one product: sum |hi||hi'| <= H_i H_j too).  The dropped
// lo.lo' term is bounded by L_i L_j (Cauchy-Schwarz); with one product the
// dropped hi.lo' + lo.hi' terms by |hi_i| L_j + L_i |hi_j| <= H_i L_j +
// L_i H_j (cross = 1).  The interval arithmetic below rounds every bound
// upwards (FP32 _ru intrinsics).
__global__ void d2_bound_kernel(CilWork w, float gam, int cross) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t np = w.n1 * w.n2;
    float lb = 0.f, ub = 0.f;
    float lbm = __int_as_float(0x7f800000), ubm = __int_as_float(0x7f800000);
    if (q < np) {
        const int64_t i = q / w.n2, j = q - i * w.n2;
        const int64_t a = i, bb = w.n1 + j;
        // segment sums of this pair, added with compensation in segment order
        float ph = 0.f, pl = 0.f;
        for (int64_t sg = 0; sg < w.S; ++sg) two_sum_acc(ph, pl, w.Ppart[sg * np + q]);
        const double P = (double)ph + (double)pl;
        const double Ni = w.N[a], Nj = w.N[bb];
        const double A = (Ni + Nj) - 2.0 * P;
        const float Af = fabsf((float)A);
        const float Ns = __fadd_ru(__fadd_ru(__double2float_ru(Ni), __double2float_ru(Nj)),
                                   __fmul_ru(2.f, fabsf(__double2float_ru(fabs(P)))));
        // Gram accumulation, dropped lo.lo, norms' compensated sums (2^-44),
        // the double rounding of A above (2^-52 of the terms)
        float dropped = __fmul_ru(w.Lf[a], w.Lf[bb]);
        if (cross)
            dropped = __fadd_ru(dropped, __fadd_ru(__fmul_ru(w.Hf[a], w.Lf[bb]), __fmul_ru(w.Lf[a], w.Hf[bb])));
        float eg = __fmul_ru(2.f, __fadd_ru(__fmul_ru(__fmul_ru(gam, w.Hf[a]), w.Hf[bb]), dropped));
        eg = __fadd_ru(eg, __fmul_ru((float)(w.dp + 64) * 5.7e-14f + 4.5e-16f, Ns));
        const float up = __fadd_ru(__double2float_ru(A), eg);
        const float D = __fadd_ru(w.Ef[a], w.Ef[bb]);
        const float er = __fmul_ru(D, __fadd_ru(__fmul_ru(2.f, __fsqrt_ru(fmaxf(up, 0.f))), D));
        float m = __fmul_ru(2.f, __fadd_ru(eg, er));
        m = __fadd_ru(m, __fmul_ru(1.2e-7f, Af)) + 1e-30f;   // FP32 rounding of A
        const float lo = __fsub_rd(__double2float_rd(A), m);
        const float hi = __fadd_ru(__double2float_ru(A), m);
        w.lo32[q] = lo;
        w.hi32[q] = hi;
        lb = fmaxf(lo, 0.f);
        ub = fmaxf(hi, 0.f);
        lbm = lb;
        ubm = ub;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lb = fmaxf(lb, __shfl_xor_sync(0xffffffffu, lb, o));
        ub = fmaxf(ub, __shfl_xor_sync(0xffffffffu, ub, o));
        lbm = fminf(lbm, __shfl_xor_sync(0xffffffffu, lbm, o));
        ubm = fminf(ubm, __shfl_xor_sync(0xffffffffu, ubm, o));
    }
    // then across the block's warps, so that one thread per block meets the
    // four global slots (same-address atomics from every warp serialised)
    __shared__ float red[4][8];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][warp] = lb;
        red[1][warp] = ub;
        red[2][warp] = lbm;
        red[3][warp] = ubm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            lb = fmaxf(lb, red[0][k]);
            ub = fmaxf(ub, red[1][k]);
            lbm = fminf(lbm, red[2][k]);
            ubm = fminf(ubm, red[3][k]);
        }
        // non-negative floats order like their bit patterns
        atomicMax(&w.scal[SC_LB1], (unsigned long long)__float_as_uint(lb));
        atomicMax(&w.scal[SC_UB1], (unsigned long long)__float_as_uint(ub));
        if (lbm < __int_as_float(0x7f800000)) {
            atomic_min_f(&w.scal[SC_LBM1], lbm);
            atomic_min_f(&w.scal[SC_UBM1], ubm);
        }
    }
}

// Threshold ranges.  Before R0 is known exactly, R0^2 lies in [lb, ub] and
// T_k = (R0 b^-k)^2 in [lb b^-2k, ub b^-2k] up to the rounding of the radius
// recursion; rel is the relative margin that covers it.  One thread per k
// (beta[k] = b^-2k from the host).  tier 1 writes FP32 ranges rounded
// outwards, tier 2 FP64 ranges.  With given radii the ranges are the exact
// thresholds.
//
// Linear law: R_k = (1 - k/M) R0 + (k/M) R_min in real arithmetic, increasing
// in both; its range follows from the ranges of R0 and R_min, widened by an
// absolute margin (the FP64 evaluation of h = (R0 - R_min)/M and
// R_k = R0 - k h errs by a few ulp of R0).
__global__ void ranges_kernel(CilWork w, const double *__restrict__ radii_in, Beta beta, int M, int tier,
                              int law) {
    const int k = threadIdx.x;
    if (k >= M) return;
    double lo, hi;
    if (radii_in) {
        lo = hi = __dmul_rn(radii_in[k], radii_in[k]);
    } else if (law_needs_min(law)) {
        double mxlo, mxhi, mnlo, mnhi;
        if (tier == 1) {
            mxlo = (double)__uint_as_float((unsigned)w.scal[SC_LB1]);
            mxhi = (double)__uint_as_float((unsigned)w.scal[SC_UB1]);
            mnlo = (double)read_min_f(w.scal[SC_LBM1]);
            mnhi = (double)read_min_f(w.scal[SC_UBM1]);
        } else {
            mxlo = __longlong_as_double((long long)w.scal[SC_LB2]);
            mxhi = __longlong_as_double((long long)w.scal[SC_UB2]);
            mnlo = read_min_d(w.scal[SC_LBM2]);
            mnhi = read_min_d(w.scal[SC_UBM2]);
        }
        const double f = (double)(k + 1) / (double)M;
        if (law == LAW_LINEAR) {
            const double r0lo = sqrt(fmax(mxlo, 0.0)), r0hi = sqrt(mxhi);
            const double rmlo = sqrt(fmax(mnlo, 0.0)), rmhi = sqrt(fmax(mnhi, 0.0));
            const double eta = (tier == 1 ? 1e-6 : 1e-13) * r0hi + 1e-300;
            const double rlo = fmax((1.0 - f) * r0lo + f * rmlo - eta, 0.0);
            const double rhi = (1.0 - f) * r0hi + f * rmhi + eta;
            lo = rlo * rlo * (1.0 - 1e-15);
            hi = rhi * rhi * (1.0 + 1e-15);
        } else {
            // fitted power law: R_k^2 = (R0^2)^(1 - f) (R_min^2)^f in real
            // arithmetic, increasing in both; the margin covers pow, the
            // bisection's b and the k divisions of the recursion
            const double rel = tier == 1 ? 1e-6 : 1e-11;
            lo = pow(fmax(mxlo, 0.0), 1.0 - f) * pow(fmax(mnlo, 0.0), f) * (1.0 - rel);
            hi = pow(fmax(mxhi, 0.0), 1.0 - f) * pow(fmax(mnhi, 0.0), f) * (1.0 + rel) + 1e-300;
        }
    } else if (tier == 1) {
        const double lb = (double)__uint_as_float((unsigned)w.scal[SC_LB1]);
        const double ub = (double)__uint_as_float((unsigned)w.scal[SC_UB1]);
        lo = lb * beta.v[k] * (1.0 - 1e-6);
        hi = ub * beta.v[k] * (1.0 + 1e-6);
    } else {
        const double lb = __longlong_as_double((long long)w.scal[SC_LB2]);
        const double ub = __longlong_as_double((long long)w.scal[SC_UB2]);
        lo = lb * beta.v[k] * (1.0 - 1e-13);
        hi = ub * beta.v[k] * (1.0 + 1e-13);
    }
    if (tier == 1) {
        w.t1lo[k] = __double2float_rd(lo);
        w.t1hi[k] = __double2float_ru(hi);
    } else {
        w.t2lo[k] = lo;
        w.t2hi[k] = hi;
    }
}

// 4a. classify: tier 1 decides, or the pair goes to tier 2 (or straight to
//     tier 3 for the exact path).
__global__ void classify1_kernel(CilWork w, const double *__restrict__ radii_in, int M, int all, int law) {
    __shared__ float tlo[32], thi[32];
    if ((int)threadIdx.x < M) {
        tlo[threadIdx.x] = w.t1lo[threadIdx.x];
        thi[threadIdx.x] = w.t1hi[threadIdx.x];
    }
    __syncthreads();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t np = w.n1 * w.n2;
    if (q >= np) return;
    w.flag[q] = 0;
    const bool lin = !radii_in && law_needs_min(law);
    if (all) {   // exact path: every pair to tier 3; all may hold the maximum (and minimum)
        unsigned long long slot = atomicAdd(&w.scal[SC_Q2], 1ull);
        w.q2[slot] = (unsigned long long)q | (radii_in ? 0ull : Q_MAX) | (lin ? Q_MIN : 0ull);
        return;
    }
    const float lo = w.lo32[q], hi = w.hi32[q];
    const bool maxc = !radii_in && hi >= __uint_as_float((unsigned)w.scal[SC_LB1]);
    const bool minc = lin && lo <= read_min_f(w.scal[SC_UBM1]);
    bool amb = false;
    for (int k = 0; k < M && !amb; ++k) amb = !(hi < tlo[k] || lo >= thi[k]);
    if (!(maxc || minc || amb)) return;
    unsigned long long slot = atomicAdd(&w.scal[SC_Q1], 1ull);
    w.q1[slot] = (unsigned long long)q | (maxc ? Q_MAX : 0ull) | (minc ? Q_MIN : 0ull);
}

// 4b. tier 2: d2 = sum (x - y)^2 from FP32 error-free transformations.
//     Per element: s = fl(x - y) and e with s + e = x - y exactly (TwoSum);
//     s^2 = p + pe exactly (product and its FMA error); 2 s e rounded
//     (error <= 2^-47 s^2); e^2 <= 2^-48 s^2 dropped.  Each thread keeps
//     four (H, L) pairs (element t into pair t mod 4 of its float4, so four
//     independent chains and 16-byte loads; unaligned rows and the last
//     d mod 4 elements into pair 0): H += p error-free (TwoSum), L
//     collects the rest in FP32: |L| <= (n + 3) 2^-24 S for n terms per pair
//     and S = sum p, so its 2n roundings cost at most 2 n (n + 4) 2^-48 S,
//     n <= ceil(d / 256) either way.  The 1024 pairs are combined in FP64
//     (error <= 1100 2^-53 of the positive sum).  The interval holds the
//     exact sum, hence (monotone rounding) its rounded value.
__device__ __forceinline__ void t2_acc(float &H, float &L, float a, float bv) {
    const float sd = a - bv;
    const float bb = sd - a;
    const float e = (a - (sd - bb)) + (-bv - bb);
    const float p = sd * sd;
    const float pe = fmaf(sd, sd, -p);
    const float cr = (2.f * sd) * e;
    two_sum_acc(H, L, p);
    L += pe + cr;
}

__global__ void __launch_bounds__(256) tier2_kernel(CilWork w, const float *__restrict__ X1, int64_t ld1,
                                                    const float *__restrict__ X2, int64_t ld2) {
    __shared__ double red[2][8];
    const unsigned long long qlen = *(volatile unsigned long long *)&w.scal[SC_Q1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (unsigned long long qi = blockIdx.x; qi < qlen; qi += gridDim.x) {
        const unsigned long long ent = w.q1[qi];
        const int64_t q = (int64_t)(ent & Q_IDX);
        const int64_t i = q / w.n2, j = q - i * w.n2;
        const float *x = X1 + i * ld1, *y = X2 + j * ld2;
        float H[4] = {0.f, 0.f, 0.f, 0.f}, L[4] = {0.f, 0.f, 0.f, 0.f};
        int64_t t0 = 0;
        if ((((uintptr_t)x | (uintptr_t)y) & 15) == 0) {
            const int64_t d4 = w.d >> 2;
            const float4 *x4 = reinterpret_cast<const float4 *>(x), *y4 = reinterpret_cast<const float4 *>(y);
#pragma unroll 4
            for (int64_t t = threadIdx.x; t < d4; t += 256) {
                const float4 a = __ldg(x4 + t), bv = __ldg(y4 + t);
                t2_acc(H[0], L[0], a.x, bv.x);
                t2_acc(H[1], L[1], a.y, bv.y);
                t2_acc(H[2], L[2], a.z, bv.z);
                t2_acc(H[3], L[3], a.w, bv.w);
            }
            t0 = d4 << 2;
        }
        for (int64_t t = t0 + threadIdx.x; t < w.d; t += 256) t2_acc(H[0], L[0], __ldg(x + t), __ldg(y + t));
        double v = ((double)H[0] + (double)L[0]) + ((double)H[1] + (double)L[1]) +
                   (((double)H[2] + (double)L[2]) + ((double)H[3] + (double)L[3]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[0][warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double D2 = 0.0;
            for (int g = 0; g < 8; ++g) D2 += red[0][g];
            const double n = (double)((w.d + 255) / 256);
            const double rel = 2.0 * (2.9e-14 + 2.0 * n * (n + 4.0) * 3.56e-15 + 1100.0 * 1.12e-16);
            const double err = rel * fabs(D2) + 1e-300;
            const double lo = D2 - err, hi = D2 + err;
            w.lo2[q] = lo;
            w.hi2[q] = hi;
            w.flag[q] = 1;
            if (ent & Q_MAX) {
                atomicMax(&w.scal[SC_LB2], (unsigned long long)__double_as_longlong(fmax(lo, 0.0)));
                atomicMax(&w.scal[SC_UB2], (unsigned long long)__double_as_longlong(fmax(hi, 0.0)));
            }
            if (ent & Q_MIN) {
                atomic_min_d(&w.scal[SC_LBM2], fmax(lo, 0.0));
                atomic_min_d(&w.scal[SC_UBM2], fmax(hi, 0.0));
            }
        }
        __syncthreads();
    }
}

// 4c. classify tier-2 pairs: those that may still hold the maximum or whose
//     tier-2 interval meets a threshold range go to tier 3.
__global__ void classify2_kernel(CilWork w, int M) {
    __shared__ double tlo[32], thi[32];
    const unsigned long long qlen = *(volatile unsigned long long *)&w.scal[SC_Q1];
    if ((unsigned long long)blockIdx.x * blockDim.x >= qlen) return;   // whole block past the queue
    if ((int)threadIdx.x < M) {
        tlo[threadIdx.x] = w.t2lo[threadIdx.x];
        thi[threadIdx.x] = w.t2hi[threadIdx.x];
    }
    __syncthreads();
    for (unsigned long long qi = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; qi < qlen;
         qi += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long ent = w.q1[qi];
        const int64_t q = (int64_t)(ent & Q_IDX);
        const double lo = w.lo2[q], hi = w.hi2[q];
        const bool maxc = (ent & Q_MAX) && hi >= __longlong_as_double((long long)w.scal[SC_LB2]);
        const bool minc = (ent & Q_MIN) && lo <= read_min_d(w.scal[SC_UBM2]);
        bool amb = false;
        for (int k = 0; k < M && !amb; ++k) amb = !(hi < tlo[k] || lo >= thi[k]);
        if (!(maxc || minc || amb)) continue;
        unsigned long long slot = atomicAdd(&w.scal[SC_Q2], 1ull);
        w.q2[slot] = (unsigned long long)q | (maxc ? Q_MAX : 0ull) | (minc ? Q_MIN : 0ull);
    }
}

// 5. tier 3: the exact value (exact.cuh) of every queued pair.
//    exact_split_kernel (queues of at most EXS_CAP pairs): one CTA per
//    (pair, segment of EXS_SEG elements); each adds its segment's exact digit
//    sums into the pair's global accumulator (integer addition, so the
//    order of the CTAs does not matter), and the pair's last CTA to arrive
//    rounds the total once.  xacc and xarr are zeroed before the launch.
__global__ void __launch_bounds__(256) exact_split_kernel(CilWork w, const float *__restrict__ X1, int64_t ld1,
                                                          const float *__restrict__ X2, int64_t ld2) {
    __shared__ XdShared<256> sh;
    const unsigned long long qlen = *(volatile unsigned long long *)&w.scal[SC_Q2];
    if (qlen > (unsigned long long)EXS_CAP) return;
    const int64_t nseg = (w.d + EXS_SEG - 1) / EXS_SEG;
    const int64_t items = (int64_t)qlen * nseg;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t slot = it / nseg, sg = it - slot * nseg;
        const unsigned long long ent = w.q2[slot];
        const int64_t q = (int64_t)(ent & Q_IDX);
        const int64_t i = q / w.n2, j = q - i * w.n2;
        const int64_t t0 = sg * EXS_SEG, len = min((int64_t)EXS_SEG, w.d - t0);
        const bool good = xd_block_digits<256>(X1 + i * ld1 + t0, X2 + j * ld2 + t0, len, sh);
        long long *acc = w.xacc + slot * XD;
        // thread k adds digit k; each fences its addition before the
        // arrival is counted
        if (threadIdx.x < XD) {
            atomicAdd((unsigned long long *)(acc + threadIdx.x), (unsigned long long)sh.tot[threadIdx.x]);
            __threadfence();
        }
        __syncthreads();   // sh.tot read; the block may reuse it
        if (threadIdx.x == 0) {
            if (!good) atomicOr(&w.xarr[EXS_CAP + slot], 1u);
            __threadfence();
            if (atomicAdd(&w.xarr[slot], 1u) == (unsigned)(nseg - 1)) {
                __threadfence();
                long long T[XD];
#pragma unroll
                for (int k = 0; k < XD; ++k) T[k] = (long long)__ldcg((const unsigned long long *)(acc + k));
                const bool bad = __ldcg(&w.xarr[EXS_CAP + slot]) != 0u;
                const double v = bad ? __longlong_as_double(0x7ff8000000000000ll) : xd_round(T);
                w.ex[q] = v;
                w.flag[q] = 2;
                if (ent & Q_MAX) atomicMax(&w.scal[SC_MAX], (unsigned long long)__double_as_longlong(v));
                if (ent & Q_MIN) atomic_min_d(&w.scal[SC_MIN], v);
            }
        }
    }
}

//    exact_kernel (longer queues): one CTA per pair (grid-stride over the
//    queue).
__global__ void __launch_bounds__(256) exact_kernel(CilWork w, const float *__restrict__ X1, int64_t ld1,
                                                    const float *__restrict__ X2, int64_t ld2) {
    __shared__ XdShared<256> sh;
    const unsigned long long qlen = *(volatile unsigned long long *)&w.scal[SC_Q2];
    if (qlen <= (unsigned long long)EXS_CAP) return;
    for (unsigned long long slot = blockIdx.x; slot < qlen; slot += gridDim.x) {
        const unsigned long long ent = w.q2[slot];
        const int64_t q = (int64_t)(ent & Q_IDX);
        const int64_t i = q / w.n2, j = q - i * w.n2;
        const double v = xd_block<256, false>(X1 + i * ld1, X2 + j * ld2, w.d, sh, nullptr);
        if (threadIdx.x == 0) {
            w.ex[q] = v;
            w.flag[q] = 2;
            if (ent & Q_MAX) atomicMax(&w.scal[SC_MAX], (unsigned long long)__double_as_longlong(v));
            if (ent & Q_MIN) atomic_min_d(&w.scal[SC_MIN], v);
        }
    }
}

// checking entry point: the exact d2 of listed pairs, one CTA per pair
__global__ void __launch_bounds__(256) exact_pairs_kernel(const float *__restrict__ X1, int64_t ld1,
                                                          const float *__restrict__ X2, int64_t ld2, int64_t d,
                                                          const int64_t *__restrict__ pairs, int64_t n,
                                                          double *__restrict__ out) {
    __shared__ XdShared<256> sh;
    for (int64_t e = blockIdx.x; e < n; e += gridDim.x) {
        const int64_t i = pairs[2 * e], j = pairs[2 * e + 1];
        const double v = xd_block<256, false>(X1 + i * ld1, X2 + j * ld2, d, sh, nullptr);
        if (threadIdx.x == 0) out[e] = v;
    }
}

// radii: R0 = sqrt(max), R_k = R_{k-1}/b, or the linear law with R_min =
// sqrt(min): h = (R0 - R_min)/M, R_k = R0 - k h  (or copy the given radii)
__global__ void radii_kernel(CilWork w, const double *__restrict__ radii_in, double b, int M, int law,
                             double *__restrict__ radii_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (radii_in) {
        radii_out[0] = __longlong_as_double(0x7ff8000000000000ll);
        for (int k = 0; k < M; ++k) radii_out[k + 1] = radii_in[k];
        return;
    }
    double R = __dsqrt_rn(__longlong_as_double((long long)w.scal[SC_MAX]));
    radii_out[0] = R;
    if (law == LAW_LINEAR) {
        const double Rm = __dsqrt_rn(read_min_d(w.scal[SC_MIN]));
        const double h = __ddiv_rn(__dsub_rn(R, Rm), (double)M);
        for (int k = 1; k <= M; ++k) radii_out[k] = __dsub_rn(R, __dmul_rn((double)k, h));
        return;
    }
    if (law == LAW_FITTED) b = fitted_b(__ddiv_rn(R, __dsqrt_rn(read_min_d(w.scal[SC_MIN]))), M);
    for (int k = 0; k < M; ++k) {
        R = __ddiv_rn(R, b);
        radii_out[k + 1] = R;
    }
}

// bins and counts: each pair is decided by the highest tier it reached.
__global__ void bins_counts_kernel(CilWork w, const double *__restrict__ radii_out, int M,
                                   uint8_t *__restrict__ bins, unsigned long long *__restrict__ counts) {
    __shared__ double Tk[32];
    __shared__ float Tlo[32], Thi[32];
    __shared__ unsigned long long cnt[32];
    if (threadIdx.x < 32) {
        cnt[threadIdx.x] = 0ull;
        if ((int)threadIdx.x < M) {
            const double r = radii_out[threadIdx.x + 1];
            const double T = __dmul_rn(r, r);
            Tk[threadIdx.x] = T;
            Tlo[threadIdx.x] = __double2float_rd(T);
            Thi[threadIdx.x] = __double2float_ru(T);
        }
    }
    __syncthreads();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t np = w.n1 * w.n2;
    int K = 0;
    if (q < np) {
        const int f = w.flag[q];
        bool und = false;
        if (f == 2) {
            const double e = w.ex[q];
            for (int k = 0; k < M; ++k) K += (e < Tk[k]) ? 1 : 0;
        } else if (f == 1) {
            const double lo = w.lo2[q], hi = w.hi2[q];
            for (int k = 0; k < M; ++k) {
                if (hi < Tk[k]) K++;
                else if (!(lo >= Tk[k])) und = true;
            }
        } else {
            const float lo = w.lo32[q], hi = w.hi32[q];
            for (int k = 0; k < M; ++k) {
                if (hi < Tlo[k]) K++;
                else if (!(lo >= Thi[k])) und = true;
            }
        }
        // cannot happen: an interval that meets a threshold was sent to the
        // next tier by the classify kernels; reported loudly if it does
        if (und) {
            atomicOr(&w.scal[SC_UNDECIDED], 1ull);
            K = 0;
        }
        bins[q] = (uint8_t)K;
    }
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < M; ++k) {
        unsigned bal = __ballot_sync(0xffffffffu, K >= k + 1);
        if (lane == 0 && bal) atomicAdd(&cnt[k], (unsigned long long)__popc(bal));
    }
    __syncthreads();
    if ((int)threadIdx.x < M && cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void finish_kernel(CilWork w, int64_t *n_rechecked, const int64_t *counts, int M, double *Cv) {
    if (blockIdx.x != 0) return;
    // -2: a Gram wait timed out; -1: a pair was left undecided; else the
    // number of pairs evaluated exactly
    if (threadIdx.x == 0 && n_rechecked)
        *n_rechecked = w.scal[SC_TIMEOUT] ? -2 : (w.scal[SC_UNDECIDED] ? -1 : (int64_t)w.scal[SC_Q2]);
    if (Cv && (int)threadIdx.x < M)
        Cv[threadIdx.x] = __ddiv_rn((double)counts[threadIdx.x], (double)w.n1 * (double)w.n2);
}

// midpoints and half-widths of the tier-1 intervals (checking entry point)
__global__ void export_approx_kernel(CilWork w, double *__restrict__ A, double *__restrict__ m) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= w.n1 * w.n2) return;
    const double lo = w.lo32[q], hi = w.hi32[q];
    A[q] = 0.5 * (lo + hi);
    m[q] = 0.5 * (hi - lo);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static rd_status check_args(int64_t ld1, int64_t n1, int64_t ld2, int64_t n2, int64_t d,
                            const double *radii_in, double b, int M, int law = LAW_POWER) {
    if (n1 < 1 || n2 < 1 || n1 > 65535 || n2 > 65535 || d < 1 || d > XD_MAX_D) return RD_ERR_INVALID_ARG;
    if (ld1 < d || ld2 < d) return RD_ERR_INVALID_ARG;
    if (M < 1 || M > 32) return RD_ERR_INVALID_ARG;
    if (!radii_in && law == LAW_POWER && !(b > 1.0)) return RD_ERR_INVALID_ARG;
    return RD_OK;
}

}  // namespace rdcil

using namespace rdcil;

extern "C" rd_status cil_workspace_size(int64_t n1, int64_t n2, int64_t d, size_t *bytes) {
    if (!bytes || n1 < 1 || n2 < 1 || d < 1) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, nullptr);
    *bytes = w.bytes;
    return RD_OK;
}

// Tensor-core accumulation model (tier 1): per chunk of cs K steps,
// np * 64 * cs / 16 instructions add into the FP32 accumulator; each adds 16
// exact bf16 products and the accumulator with at most 17 roundings of
// 2^-23 relative to the magnitudes involved.  Within a segment the kernel
// adds its m = nchunk / S chunk partials into a plain FP32 running sum: m - 1
// roundings of at most 2^-24 of the running magnitude, bounded by
// m 2^-24 (1.01) of the magnitudes (the partials' own accumulation errors
// are far below the 1 %).  The S segment sums are then added with TwoSum
// into an FP32 hi/lo pair: for n terms that errs by at most about (n u)^2
// of their magnitudes (u = 2^-24), taken here as (S + 4)^2 2^-47.
static float gram_gamma(const CilWork &w) {
    const double m = (double)(w.nchunk / w.S);
    const double n = (double)(w.S + 4);
    const double g = ((double)w.np_ * 64.0 * (double)w.cs / 16.0 + 1.0) * 17.0 * 1.1920928955078125e-7 +
                     m * 5.9604644775390625e-8 * 1.01 + n * n * 7.105427357601002e-15;
    return (float)(g * (1.0 + 1e-6));
}

// pack + tensor-core Gram + tier-1 intervals
static rd_status tier1(const CilWork &w, const float *X1, int64_t ld1, const float *X2, int64_t ld2,
                       cudaStream_t s) {
    const int64_t n1 = w.n1, n2 = w.n2, np = n1 * n2;
    centre_kernel<<<(unsigned)((w.dp + 255) / 256), 256, 0, s>>>(X1, ld1, n1, X2, ld2, n2, w.d, w.dp, w.centre);
    note_launch();
    pack_kernel<<<(unsigned)(n1 + n2), 256, 0, s>>>(X1, ld1, n1, X2, ld2, w.d, w.dp, w.centre, w.hi,
                                                    w.np_ == 3 ? w.lo : nullptr, w.N, w.H, w.L, w.E, w.Hf, w.Lf,
                                                    w.Ef);
    note_launch();
    rd_status st = launch_gram_tc(w.hi, w.lo, n1, n2, w.dp, w.S, w.cs, (int)w.np_, w.Ppart,
                                  reinterpret_cast<uint32_t *>(&w.scal[SC_TIMEOUT]), s);
    if (st) return st;
    d2_bound_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(w, gram_gamma(w), w.np_ == 1 ? 1 : 0);
    note_launch();
    return RD_OK;
}

// Internal entry for the multi-feature correlation integral: tier-1
// intervals [lo, hi] (FP32, outward) of the exact squared distance of
// every pair of two pattern arrays, left in the workspace; *timeout points
// at the word the tensor-core stage raises on a timeout.
rd_status cil_tier1_intervals(const float *X1, int64_t ld1, int64_t n1, const float *X2, int64_t ld2, int64_t n2,
                              int64_t d, void *work, size_t work_bytes, const float **lo, const float **hi,
                              const unsigned long long **timeout, cudaStream_t s) {
    if (n1 < 1 || n2 < 1 || n1 > 65535 || n2 > 65535 || d < 1 || d > XD_MAX_D || ld1 < d || ld2 < d)
        return RD_ERR_INVALID_ARG;
    if (!X1 || !X2 || !work || (((uintptr_t)work & 255) != 0)) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    RD_CUDA_TRY(cudaMemsetAsync(w.scal, 0, 16 * sizeof(unsigned long long), s));
    rd_status st = tier1(w, X1, ld1, X2, ld2, s);
    if (st) return st;
    *lo = w.lo32;
    *hi = w.hi32;
    *timeout = &w.scal[SC_TIMEOUT];
    return RD_OK;
}

static rd_status cil_run(const float *X1, int64_t ld1, int64_t n1, const float *X2, int64_t ld2, int64_t n2,
                         int64_t d, const double *radii_in, double b, int32_t M, double *radii_out,
                         uint8_t *bins, int64_t *counts, double *Cv, int64_t *n_rechecked, void *work,
                         size_t work_bytes, void *stream, bool exact, int law = LAW_POWER) {
    rd_status st = check_args(ld1, n1, ld2, n2, d, radii_in, b, M, law);
    if (st) return st;
    if (!X1 || !X2 || !radii_out || !bins || !counts || !work) return RD_ERR_INVALID_ARG;
    if (((uintptr_t)work & 255) != 0) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = n1 * n2;
    const unsigned gp = (unsigned)((np + 255) / 256);
    RD_CUDA_TRY(cudaMemsetAsync(w.scal, 0, 16 * sizeof(unsigned long long), s));
    RD_CUDA_TRY(cudaMemsetAsync(counts, 0, M * sizeof(int64_t), s));
    if (!exact) {
        st = tier1(w, X1, ld1, X2, ld2, s);
        if (st) return st;
    }
    Beta beta{};
    {
        double f = 1.0;
        for (int k = 0; k < M; ++k) {
            f = law == LAW_POWER ? f / (b * b) : 0.0;
            beta.v[k] = radii_in ? 0.0 : f;
        }
    }
    if (!exact) {
        ranges_kernel<<<1, 32, 0, s>>>(w, radii_in, beta, M, 1, law);
        note_launch();
    }
    classify1_kernel<<<gp, 256, 0, s>>>(w, radii_in, M, exact ? 1 : 0, law);
    note_launch();
    if (!exact) {
        // one CTA per queued pair at a time; the tier waits on memory, so
        // six CTAs per SM (what its 40 registers allow) keep more rows in
        // flight than two (2 x 1024 x 32768: 0.52 against 0.57 ms for the
        // whole correlation integral); the sum order is per pair, so the
        // grid does not change results
        const unsigned g2 = (unsigned)(np < 6 * N_SM ? np : 6 * N_SM);
        tier2_kernel<<<g2, 256, 0, s>>>(w, X1, ld1, X2, ld2);
        note_launch();
        ranges_kernel<<<1, 32, 0, s>>>(w, radii_in, beta, M, 2, law);
        note_launch();
        // the queue is short: blocks past it exit before loading anything
        classify2_kernel<<<(gp < 8 * N_SM ? gp : 8 * N_SM), 256, 0, s>>>(w, M);
        note_launch();
    }
    {
        RD_CUDA_TRY(cudaMemsetAsync(w.xacc, 0, sizeof(long long) * EXS_CAP * XD + sizeof(unsigned) * 2 * EXS_CAP,
                                    s));
        exact_split_kernel<<<2 * N_SM, 256, 0, s>>>(w, X1, ld1, X2, ld2);
        note_launch();
        const unsigned g3 = (unsigned)(np < 2 * N_SM ? np : 2 * N_SM);
        exact_kernel<<<g3, 256, 0, s>>>(w, X1, ld1, X2, ld2);
        note_launch();
    }
    radii_kernel<<<1, 32, 0, s>>>(w, radii_in, b, M, law, radii_out);
    note_launch();
    bins_counts_kernel<<<gp, 256, 0, s>>>(w, radii_out, M, bins, (unsigned long long *)counts);
    note_launch();
    finish_kernel<<<1, 32, 0, s>>>(w, n_rechecked, counts, M, Cv);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// Checking entry point: the tier-1 approximation of every pair as midpoint A
// and half-width m of its interval (pack + tensor-core Gram + bound, before
// any exact evaluation).  |A - d2| <= m must hold for every pair.
extern "C" rd_status cil_debug_approx(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2,
                                      int64_t n2, int64_t d, double *d_A, double *d_m, void *d_work,
                                      size_t work_bytes, void *stream) {
    rd_status st = check_args(ld1, n1, ld2, n2, d, nullptr, 2.0, 1);
    if (st) return st;
    if (!d_X1 || !d_X2 || !d_A || !d_m || !d_work || (((uintptr_t)d_work) & 255)) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, d_work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = n1 * n2;
    RD_CUDA_TRY(cudaMemsetAsync(w.scal, 0, 16 * sizeof(unsigned long long), s));
    st = tier1(w, d_X1, ld1, d_X2, ld2, s);
    if (st) return st;
    export_approx_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(w, d_A, d_m);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// Benchmarking entry point: re-run only the tensor-core Gram stage on a
// workspace that a previous cil_features / cil_debug_approx call with the
// same (n1, n2, d) has packed.  Returns the FLOP count of the launch in
// *flops (3 bf16 products per element pair, 2 flops each).
extern "C" rd_status cil_gram_only(int64_t n1, int64_t n2, int64_t d, void *d_work, size_t work_bytes,
                                   double *flops, void *stream) {
    if (n1 < 1 || n2 < 1 || d < 1 || !d_work || (((uintptr_t)d_work) & 255)) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, d_work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    if (flops) *flops = (double)w.np_ * 2.0 * (double)n1 * (double)n2 * (double)w.dp;
    return launch_gram_tc(w.hi, w.lo, n1, n2, w.dp, w.S, w.cs, (int)w.np_, w.Ppart,
                          reinterpret_cast<uint32_t *>(&w.scal[SC_TIMEOUT]), (cudaStream_t)stream);
}

extern "C" rd_status cil_set_gram_products(int32_t mode) {
    if (mode != 0 && mode != 1 && mode != 3) return RD_ERR_INVALID_ARG;
    g_gram_products.store(mode == 0 ? 3 : mode);
    return RD_OK;
}

extern "C" rd_status cil_queue_lengths(int64_t n1, int64_t n2, int64_t d, const void *d_work, size_t work_bytes,
                                      int64_t *d_out, void *stream) {
    if (n1 < 1 || n2 < 1 || d < 1 || !d_work || !d_out || (((uintptr_t)d_work) & 255)) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, const_cast<void *>(d_work));
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    static_assert(SC_Q2 == SC_Q1 + 1, "adjacent queue slots");
    RD_CUDA_TRY(cudaMemcpyAsync(d_out, &w.scal[SC_Q1], 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
    return RD_OK;
}

extern "C" int32_t cil_gram_products(int64_t n1, int64_t n2, int64_t d) {
    if (n1 < 1 || n2 < 1 || d < 1) return -1;
    return (int32_t)layout(n1, n2, d, nullptr).np_;
}

extern "C" rd_status cil_features(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2,
                                  int64_t n2, int64_t d, const double *d_radii_in, double b, int32_t M,
                                  double *d_radii_out, uint8_t *d_bins, int64_t *d_counts, double *d_C,
                                  int64_t *d_n_rechecked, void *d_work, size_t work_bytes, void *stream) {
    return cil_run(d_X1, ld1, n1, d_X2, ld2, n2, d, d_radii_in, b, M, d_radii_out, d_bins, d_counts, d_C,
                   d_n_rechecked, d_work, work_bytes, stream, false);
}

extern "C" rd_status cil_features_linear(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                         int64_t ld2, int64_t n2, int64_t d, int32_t M, double *d_radii_out,
                                         uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_rechecked,
                                         void *d_work, size_t work_bytes, void *stream) {
    return cil_run(d_X1, ld1, n1, d_X2, ld2, n2, d, nullptr, 0.0, M, d_radii_out, d_bins, d_counts, d_C,
                   d_n_rechecked, d_work, work_bytes, stream, false, LAW_LINEAR);
}

extern "C" rd_status cil_features_fitted(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                         int64_t ld2, int64_t n2, int64_t d, int32_t M, double *d_radii_out,
                                         uint8_t *d_bins, int64_t *d_counts, double *d_C, int64_t *d_n_rechecked,
                                         void *d_work, size_t work_bytes, void *stream) {
    return cil_run(d_X1, ld1, n1, d_X2, ld2, n2, d, nullptr, 0.0, M, d_radii_out, d_bins, d_counts, d_C,
                   d_n_rechecked, d_work, work_bytes, stream, false, LAW_FITTED);
}

extern "C" rd_status cil_exact_d2(const float *d_X1, int64_t ld1, const float *d_X2, int64_t ld2, int64_t d,
                                  const int64_t *d_pairs, int64_t n_pairs, double *d_out, void *stream) {
    if (d < 1 || d > XD_MAX_D || ld1 < d || ld2 < d || n_pairs < 0) return RD_ERR_INVALID_ARG;
    if (n_pairs == 0) return RD_OK;
    if (!d_X1 || !d_X2 || !d_pairs || !d_out) return RD_ERR_INVALID_ARG;
    const unsigned g = (unsigned)(n_pairs < 4 * N_SM ? n_pairs : 4 * N_SM);
    exact_pairs_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(d_X1, ld1, d_X2, ld2, d, d_pairs, n_pairs, d_out);
    note_launch();
    return cuda_status(cudaGetLastError());
}

extern "C" rd_status cil_features_exact(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                        int64_t ld2, int64_t n2, int64_t d, const double *d_radii_in, double b,
                                        int32_t M, double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                                        double *d_C, void *d_work, size_t work_bytes, void *stream) {
    return cil_run(d_X1, ld1, n1, d_X2, ld2, n2, d, d_radii_in, b, M, d_radii_out, d_bins, d_counts, d_C,
                   nullptr, d_work, work_bytes, stream, true);
}

// ===========================================================================
// Allocation-free variant of cil_features.
//
// Some callers cannot call cudaMalloc on the hot path: cudaMalloc may
// synchronise the whole device (stalling every other stream of a sampler
// that overlaps model runs with likelihood evaluations), and hosts that own
// a fixed device-memory budget through their own pool allocator do not let
// plug-in code allocate outside it.  This entry point needs no workspace
// from the caller: its scratch is one file-scope device array of
// CIL_STATIC_BYTES, held by every GPU that loads the library until the
// process exits.
// ===========================================================================
#include <mutex>

namespace rdcil {
static constexpr size_t CIL_STATIC_BYTES = 16u << 20;     // 16 MiB per device
static constexpr int64_t CIL_STATIC_MAX_N = 128;          // patterns per set
static constexpr int64_t CIL_STATIC_MAX_D = 8192;         // pattern length
static __device__ __align__(256) unsigned char g_cil_static_scratch[CIL_STATIC_BYTES];

// Device address of the array, looked up once per device with that device
// current (in host code the array's name is only a host-side stand-in).
static void *static_scratch_ptr(int device, rd_status &st) {
    static std::mutex mu;
    static void *ptrs[64] = {nullptr};
    st = RD_OK;
    if (device < 0 || device >= 64) { st = RD_ERR_UNSUPPORTED; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cil_static_scratch) != cudaSuccess || !p) {
            st = RD_ERR_CUDA;
            return nullptr;
        }
        ptrs[device] = p;
    }
    return ptrs[device];
}
}  // namespace rdcil

extern "C" rd_status cil_features_static(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2,
                                         int64_t ld2, int64_t n2, int64_t d, const double *d_radii_in, double b,
                                         int32_t M, double *d_radii_out, uint8_t *d_bins, int64_t *d_counts,
                                         double *d_C, int64_t *d_n_rechecked, void *stream) {
    if (n1 > CIL_STATIC_MAX_N || n2 > CIL_STATIC_MAX_N || d > CIL_STATIC_MAX_D) return RD_ERR_INVALID_ARG;
    if (n1 < 1 || n2 < 1 || d < 1) return RD_ERR_INVALID_ARG;
    if (layout(n1, n2, d, nullptr).bytes > CIL_STATIC_BYTES) return RD_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return RD_ERR_CUDA;
    rd_status st;
    void *scratch = static_scratch_ptr(dev, st);
    if (st) return st;
    return cil_features(d_X1, ld1, n1, d_X2, ld2, n2, d, d_radii_in, b, M, d_radii_out, d_bins, d_counts, d_C,
                        d_n_rechecked, scratch, CIL_STATIC_BYTES, stream);
}
