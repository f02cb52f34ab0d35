// Correlation integral of two pattern sets (eq. eCDF, eq. CIL, Sec. 2.1).
//
// Exactness contract.  For every pair the library decides K_ij =
// #{k : d2_ij < R_k^2} for the canonical d2_ij = sum_t (x_t - y_t)^2
// evaluated in FP64 in one fixed order (term t into partial t mod 256, each
// partial in increasing t, partials combined by a halving tree within groups
// of 32 and then across the 8 groups; no FMA).  It does so in three stages:
//   1. pack:  centre every pattern by the set mean c (translation does not
//      change distances), split x - c into bf16 hi + lo, and record per
//      pattern N = |hi+lo|^2, H = |hi| + |lo|, L = |lo| and the
//      representation error E = |(x - c) - (hi + lo)| (all FP64);
//   2. Gram:  P_ij = hi_i.hi_j + hi_i.lo_j + lo_i.hi_j (bf16 products, FP32
//      accumulation per K-chunk, chunks summed in FP64);
//   3. bound: A = N_i + N_j - 2 P_ij approximates d2_ij with a rigorous error
//      bound built from the FP32 accumulation model, the dropped lo.lo term,
//      E_i + E_j and the rounding of the canonical sum.  A pair whose interval
//      [A - m, A + m] contains a threshold (or could hold the maximum that
//      defines R0) is re-evaluated with the canonical sum.
// Counts per radius are reduced with warp ballot + popc.
#include <cstdio>
#include <cuda_bf16.h>
#include "common.cuh"

namespace rdcil {

rd_status launch_gram_tc(const void *hi, const void *lo, int64_t n1, int64_t n2, int64_t dp, int64_t kc,
                         int64_t nchunk, float *Ppart, uint32_t *status, cudaStream_t s);

static constexpr int KCHUNK_MAX = 512;   // longest split-K chunk (bounds FP32 accumulation error)
static constexpr int PAD = 64;           // padded pattern length granularity
static constexpr int TILE = 64;          // Gram output tile (pairs per side)

static inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

struct CilWork {
    int64_t n1, n2, d, dp, kc, nchunk;
    float *centre;          // [dp]
    __nv_bfloat16 *hi;      // [(n1+n2)][dp]
    __nv_bfloat16 *lo;      // [(n1+n2)][dp]
    double *N, *H, *L, *E;  // [(n1+n2)]
    float *Ppart;           // [nchunk][n1][n2]
    double *A, *Mg;         // [n1*n2] approximate d2 and its error bound (Mg < 0: A is exact)
    unsigned long long *queue; // [n1*n2] pairs to evaluate exactly (bit 63: may hold the maximum)
    unsigned long long *scal;  // [0] max lower bound, [1] max upper bound, [2] exact max (FP64 bits),
                               // [3] n_rechecked, [4] queue length
    size_t bytes;
};

static CilWork layout(int64_t n1, int64_t n2, int64_t d, void *base) {
    CilWork w{};
    w.n1 = n1; w.n2 = n2; w.d = d;
    w.dp = round_up(d, PAD);
    // split-K chunk: enough CTAs to cover the GPU twice, at most KCHUNK_MAX
    int64_t tiles = ((n1 + TILE - 1) / TILE) * ((n2 + TILE - 1) / TILE);
    int64_t want = (2 * 148 + tiles - 1) / tiles;
    int64_t kc = round_up((w.dp + want - 1) / want, PAD);
    if (kc > KCHUNK_MAX) kc = KCHUNK_MAX;
    w.kc = kc;
    w.nchunk = (w.dp + kc - 1) / kc;
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
    w.Ppart = (float *)take(sizeof(float) * w.nchunk * n1 * n2);
    w.A = (double *)take(sizeof(double) * n1 * n2);
    w.Mg = (double *)take(sizeof(double) * n1 * n2);
    w.queue = (unsigned long long *)take(sizeof(unsigned long long) * n1 * n2);
    w.scal = (unsigned long long *)take(sizeof(unsigned long long) * 8);
    w.bytes = off;
    return w;
}

// ---------------------------------------------------------------------------
// canonical distance: sequential FP64, no FMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sq_diff(float a, float b) {
    double df = __dsub_rn((double)a, (double)b);
    return __dmul_rn(df, df);
}

// Canonical d2 of one pair by a whole 256-thread block, in the fixed order
// above.  FP64 has a long dependent-operation latency on this GPU, so the
// order is chosen for a short dependency chain: d/256 + 8 additions.
// Result valid in thread 0; sw = 8 doubles of shared memory.
__device__ double canonical_block(const float *__restrict__ x, const float *__restrict__ y, int64_t d,
                                  double *sw) {
    const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
    double acc = 0.0;
    for (int64_t t = j; t < d; t += 256) acc = __dadd_rn(acc, sq_diff(__ldg(x + t), __ldg(y + t)));
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, s));
    if (lane == 0) sw[warp] = acc;
    __syncthreads();
    double r = 0.0;
    if (j == 0) {
        double w[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) w[g] = sw[g];
#pragma unroll
        for (int s = 4; s >= 1; s >>= 1)
#pragma unroll
            for (int i = 0; i < s; ++i) w[i] = __dadd_rn(w[i], w[i + s]);
        r = w[0];
    }
    __syncthreads();
    return r;
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
    // keeps |x - c| small so the bf16 split loses little
    float s = 0.f;
    for (int64_t i = 0; i < n1; ++i) s += X1[i * ld1 + t];
    for (int64_t j = 0; j < n2; ++j) s += X2[j * ld2 + t];
    centre[t] = s / (float)(n1 + n2);
}

__global__ void pack_kernel(const float *__restrict__ X1, int64_t ld1, int64_t n1,
                            const float *__restrict__ X2, int64_t ld2, int64_t d, int64_t dp,
                            const float *__restrict__ centre, __nv_bfloat16 *__restrict__ hi,
                            __nv_bfloat16 *__restrict__ lo, double *__restrict__ Nn, double *__restrict__ Hn,
                            double *__restrict__ Ln, double *__restrict__ En) {
    const int64_t i = blockIdx.x;
    const float *x = i < n1 ? X1 + i * ld1 : X2 + (i - n1) * ld2;
    // N = |hi + lo|^2 to ~2^-44 relative (compensated FP32); H, L, E are
    // upper bounds (plain FP32 sums, inflated below)
    float nh = 0.f, nl = 0.f, sH = 0.f, sL = 0.f, sE = 0.f;
    for (int64_t t = threadIdx.x; t < dp; t += blockDim.x) {
        __nv_bfloat16 h = __float2bfloat16_rn(0.f), l = __float2bfloat16_rn(0.f);
        if (t < d) {
            float xv = x[t], cv = centre[t];
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
            two_sum_acc(nh, nl, p);
            nl += pe;
            sH = fmaf(hf, hf, sH);
            sL = fmaf(lf, lf, sL);
            float e = fabsf(dc) + fabsf(r - lf);   // |(x - c) - (hi + lo)|, bounded
            sE = fmaf(e, e, sE);
        }
        hi[i * dp + t] = h;
        lo[i * dp + t] = l;
    }
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
    }
}

// ---------------------------------------------------------------------------
// 2. Gram product: tensor cores (gram_tc.cu), split-K chunks of kc.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// 3a. approximate d2 and its rigorous error bound; running max lower bound
// ---------------------------------------------------------------------------
// Accumulation model for the Gram: a sequence of n roundings into one FP32
// accumulator errs by at most n * u * S, S = sum of the magnitudes of the
// products, u the unit roundoff of one accumulation step (gam = n * u is
// passed in per Gram kernel).  Here S = sum |hi||hi'| + |hi||lo'| + |lo||hi'|
// <= H_i H_j.  The dropped lo.lo' term is bounded by L_i L_j.
__device__ __forceinline__ void approx_and_bound(const CilWork &w, int64_t i, int64_t j, double P,
                                                 double gam, double &A, double &m) {
    const int64_t a = i, b = w.n1 + j;
    const double Ni = w.N[a], Nj = w.N[b];
    A = (Ni + Nj) - 2.0 * P;
    // N_i, N_j carry <= (dp + 64) 2^-44 relative error (compensated FP32)
    double eg = 2.0 * (gam * w.H[a] * w.H[b] + w.L[a] * w.L[b]) +
                4.0 * (double)(w.dp + 64) * 5.684341886080802e-14 * (Ni + Nj + 2.0 * fabs(P));
    double up = fmax(A + eg, 0.0);
    double D = w.E[a] + w.E[b];
    double er = D * (2.0 * sqrt(up) + D);
    double ec = (double)(w.d + 8) * 2.220446049250313e-16 * (up + er);
    m = 2.0 * (eg + er + ec) + 1e-300;
}

__global__ void d2_bound_kernel(CilWork w, double gam) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t np = w.n1 * w.n2;
    double lb = 0.0, ub = 0.0;
    if (q < np) {
        int64_t i = q / w.n2, j = q - i * w.n2;
        float ph = 0.f, pl = 0.f;
        for (int64_t c = 0; c < w.nchunk; ++c) two_sum_acc(ph, pl, w.Ppart[c * np + q]);
        double P = (double)ph + (double)pl;
        double A, m;
        approx_and_bound(w, i, j, P, gam, A, m);
        w.A[q] = A;
        w.Mg[q] = m;
        lb = fmax(A - m, 0.0);
        ub = fmax(A + m, 0.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lb = fmax(lb, __shfl_xor_sync(0xffffffffu, lb, o));
        ub = fmax(ub, __shfl_xor_sync(0xffffffffu, ub, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(&w.scal[0], (unsigned long long)__double_as_longlong(lb));
        atomicMax(&w.scal[1], (unsigned long long)__double_as_longlong(ub));
    }
}

// 3b. exact pass.  classify_kernel enqueues every pair that could hold the
//     maximum (upper bound >= the largest lower bound) or whose interval
//     could contain a threshold.  Before R0 is known exactly, R0^2 lies in
//     [lbmax, ubmax], so T_k = (R0 b^-k)^2 lies in [lbmax b^-2k, ubmax b^-2k]
//     up to the rounding of the radius recursion (relative 1e-13 margin).
//     canonical_kernel then evaluates the queued pairs (one block each) and
//     overwrites A with the exact value, Mg = -1 as the flag.
__global__ void classify_kernel(CilWork w, const double *__restrict__ radii_in, double b, int M, int all) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t np = w.n1 * w.n2;
    if (q >= np) return;
    bool need = all != 0, maxc = false;
    if (!radii_in) {
        const double lbmax = __longlong_as_double((long long)w.scal[0]);
        const double ubmax = __longlong_as_double((long long)w.scal[1]);
        const double lo = all ? 0.0 : w.A[q] - w.Mg[q], hi = all ? 1.0 : w.A[q] + w.Mg[q];
        maxc = all || hi >= lbmax;
        need = need || maxc;
        double f = 1.0;
        for (int k = 0; k < M && !need; ++k) {
            f = f / (b * b);
            double tlo = lbmax * f * (1.0 - 1e-13), thi = ubmax * f * (1.0 + 1e-13);
            need = !(hi < tlo || lo > thi);
        }
    } else if (!need) {
        const double lo = w.A[q] - w.Mg[q], hi = w.A[q] + w.Mg[q];
        for (int k = 0; k < M && !need; ++k) {
            double T = __dmul_rn(radii_in[k], radii_in[k]);
            need = !(hi < T || lo >= T);
        }
    }
    if (!need) return;
    unsigned long long slot = atomicAdd(&w.scal[4], 1ull);
    w.queue[slot] = (unsigned long long)q | (maxc ? (1ull << 63) : 0ull);
}

__global__ void __launch_bounds__(256) canonical_kernel(CilWork w, const float *__restrict__ X1, int64_t ld1,
                                                        const float *__restrict__ X2, int64_t ld2, int count) {
    __shared__ double sw[8];
    const unsigned long long qlen = *(volatile unsigned long long *)&w.scal[4];
    for (unsigned long long qi = blockIdx.x; qi < qlen; qi += gridDim.x) {
        const unsigned long long ent = w.queue[qi];
        const int64_t q = (int64_t)(ent & ~(1ull << 63));
        const int64_t i = q / w.n2, j = q - i * w.n2;
        double e = canonical_block(X1 + i * ld1, X2 + j * ld2, w.d, sw);
        if (threadIdx.x == 0) {
            w.A[q] = e;
            w.Mg[q] = -1.0;
            if (ent >> 63) atomicMax(&w.scal[2], (unsigned long long)__double_as_longlong(e));
            if (count) atomicAdd(&w.scal[3], 1ull);
        }
    }
}

// 3c. radii: R0 = sqrt(max), R_k = R_{k-1}/b  (or copy the given radii)
__global__ void radii_kernel(CilWork w, const double *__restrict__ radii_in, double b, int M,
                             double *__restrict__ radii_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (radii_in) {
        radii_out[0] = __longlong_as_double(0x7ff8000000000000ll);
        for (int k = 0; k < M; ++k) radii_out[k + 1] = radii_in[k];
        return;
    }
    double R = __dsqrt_rn(__longlong_as_double((long long)w.scal[2]));
    radii_out[0] = R;
    for (int k = 0; k < M; ++k) {
        R = __ddiv_rn(R, b);
        radii_out[k + 1] = R;
    }
}

// 3d. bins and counts.  A pair is classified from [A - m, A + m] when no
//     threshold T_k = R_k*R_k falls inside; otherwise from the canonical sum.
__global__ void bins_counts_kernel(CilWork w, const double *__restrict__ radii_out, int M,
                                   uint8_t *__restrict__ bins, unsigned long long *__restrict__ counts) {
    __shared__ double Tk[32];
    __shared__ unsigned long long cnt[32];
    if (threadIdx.x < 32) {
        cnt[threadIdx.x] = 0ull;
        if ((int)threadIdx.x < M) {
            double r = radii_out[threadIdx.x + 1];
            Tk[threadIdx.x] = __dmul_rn(r, r);
        }
    }
    __syncthreads();
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t np = w.n1 * w.n2;
    int K = 0;
    if (q < np) {
        bool amb = false;
        {
            const double A = w.A[q], m = w.Mg[q];
            if (m < 0.0) {
                for (int k = 0; k < M; ++k) K += (A < Tk[k]) ? 1 : 0;
            } else {
                for (int k = 0; k < M; ++k) {
                    double T = Tk[k];
                    if (A + m < T) K++;
                    else if (!(A - m >= T)) amb = true;
                }
            }
        }
        // A pair the exact pass did not foresee cannot occur (its interval would
        // straddle a threshold inside the predicted range); flag it loudly.
        if (amb) {
            K = 0xFF;
            atomicOr(&w.scal[5], 1ull);
        }
        bins[q] = (uint8_t)K;
    }
    const int lane = threadIdx.x & 31;
    if (K == 0xFF) K = 0;
    for (int k = 0; k < M; ++k) {
        unsigned bal = __ballot_sync(0xffffffffu, K >= k + 1);
        if (lane == 0 && bal) atomicAdd(&cnt[k], (unsigned long long)__popc(bal));
    }
    __syncthreads();
    if ((int)threadIdx.x < M && cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void finish_kernel(CilWork w, int64_t *n_rechecked, const int64_t *counts, int M, double *Cv) {
    if (blockIdx.x != 0) return;
    // a set scal[5] (unforeseen ambiguous pair) reports -1 rechecks, a Gram
    // timeout (scal[6]) -2
    if (threadIdx.x == 0 && n_rechecked)
        *n_rechecked = w.scal[6] ? -2 : (w.scal[5] ? -1 : (int64_t)w.scal[3]);
    if (Cv && (int)threadIdx.x < M)
        Cv[threadIdx.x] = __ddiv_rn((double)counts[threadIdx.x], (double)w.n1 * (double)w.n2);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static rd_status check_args(int64_t ld1, int64_t n1, int64_t ld2, int64_t n2, int64_t d,
                            const double *radii_in, double b, int M) {
    if (n1 < 1 || n2 < 1 || n1 > 65535 || n2 > 65535 || d < 1) return RD_ERR_INVALID_ARG;
    if (ld1 < d || ld2 < d) return RD_ERR_INVALID_ARG;
    if (M < 1 || M > 32) return RD_ERR_INVALID_ARG;
    if (!radii_in && !(b > 1.0)) return RD_ERR_INVALID_ARG;
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

static rd_status cil_run(const float *X1, int64_t ld1, int64_t n1, const float *X2, int64_t ld2, int64_t n2,
                         int64_t d, const double *radii_in, double b, int32_t M, double *radii_out,
                         uint8_t *bins, int64_t *counts, double *Cv, int64_t *n_rechecked, void *work,
                         size_t work_bytes, void *stream, bool exact) {
    rd_status st = check_args(ld1, n1, ld2, n2, d, radii_in, b, M);
    if (st) return st;
    if (!X1 || !X2 || !radii_out || !bins || !counts || !work) return RD_ERR_INVALID_ARG;
    if (((uintptr_t)work & 255) != 0) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t np = n1 * n2;
    unsigned gp = (unsigned)((np + 255) / 256);
    RD_CUDA_TRY(cudaMemsetAsync(w.scal, 0, 8 * sizeof(unsigned long long), s));
    RD_CUDA_TRY(cudaMemsetAsync(counts, 0, M * sizeof(int64_t), s));
    if (!exact) {
        centre_kernel<<<(unsigned)((w.dp + 255) / 256), 256, 0, s>>>(X1, ld1, n1, X2, ld2, n2, d, w.dp, w.centre);
        note_launch();
        pack_kernel<<<(unsigned)(n1 + n2), 256, 0, s>>>(X1, ld1, n1, X2, ld2, d, w.dp, w.centre, w.hi, w.lo, w.N,
                                                        w.H, w.L, w.E);
        note_launch();
        st = launch_gram_tc(w.hi, w.lo, n1, n2, w.dp, w.kc, w.nchunk, w.Ppart,
                            reinterpret_cast<uint32_t *>(&w.scal[6]), s);
        if (st) return st;
        // Tensor-core accumulation model: per chunk 3*kc/16 instructions add
        // into the FP32 accumulator; each adds 16 exact bf16 products and
        // the accumulator with at most 17 roundings of 2^-23 relative to the
        // magnitudes involved.  The chunk partials are summed by a
        // compensated FP32 sum ((nchunk + 4) 2^-45 of the magnitudes).
        const double gam = (3.0 * (double)w.kc / 16.0 + 1.0) * 17.0 * 1.1920928955078125e-7 +
                           (double)(w.nchunk + 4) * 2.842170943040401e-14;
        d2_bound_kernel<<<gp, 256, 0, s>>>(w, gam);
        note_launch();
    }
    classify_kernel<<<gp, 256, 0, s>>>(w, radii_in, b, M, exact ? 1 : 0);
    note_launch();
    {
        int64_t ncta = 2 * 148;
        if (ncta > np) ncta = np;
        canonical_kernel<<<(unsigned)ncta, 256, 0, s>>>(w, X1, ld1, X2, ld2, exact ? 0 : 1);
        note_launch();
    }
    radii_kernel<<<1, 32, 0, s>>>(w, radii_in, b, M, radii_out);
    note_launch();
    bins_counts_kernel<<<gp, 256, 0, s>>>(w, radii_out, M, bins, (unsigned long long *)counts);
    note_launch();
    finish_kernel<<<1, 32, 0, s>>>(w, n_rechecked, counts, M, Cv);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// Checking entry point: the approximate d2 (A) and its error bound (m) of
// every pair from the pack + tensor-core Gram stages, before any exact
// evaluation.  |A - canonical d2| <= m must hold for every pair.
extern "C" rd_status cil_debug_approx(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2,
                                      int64_t n2, int64_t d, double *d_A, double *d_m, void *d_work,
                                      size_t work_bytes, void *stream) {
    rd_status st = check_args(ld1, n1, ld2, n2, d, nullptr, 2.0, 1);
    if (st) return st;
    if (!d_X1 || !d_X2 || !d_A || !d_m || !d_work || (((uintptr_t)d_work) & 255)) return RD_ERR_INVALID_ARG;
    CilWork w = layout(n1, n2, d, d_work);
    if (w.bytes > work_bytes) return RD_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t np = n1 * n2;
    RD_CUDA_TRY(cudaMemsetAsync(w.scal, 0, 8 * sizeof(unsigned long long), s));
    centre_kernel<<<(unsigned)((w.dp + 255) / 256), 256, 0, s>>>(d_X1, ld1, n1, d_X2, ld2, n2, d, w.dp, w.centre);
    note_launch();
    pack_kernel<<<(unsigned)(n1 + n2), 256, 0, s>>>(d_X1, ld1, n1, d_X2, ld2, d, w.dp, w.centre, w.hi, w.lo, w.N,
                                                    w.H, w.L, w.E);
    note_launch();
    st = launch_gram_tc(w.hi, w.lo, n1, n2, w.dp, w.kc, w.nchunk, w.Ppart,
                        reinterpret_cast<uint32_t *>(&w.scal[6]), s);
    if (st) return st;
    const double gam = (3.0 * (double)w.kc / 16.0 + 1.0) * 17.0 * 1.1920928955078125e-7 +
                       (double)(w.nchunk + 4) * 2.842170943040401e-14;
    d2_bound_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(w, gam);
    note_launch();
    RD_CUDA_TRY(cudaMemcpyAsync(d_A, w.A, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RD_CUDA_TRY(cudaMemcpyAsync(d_m, w.Mg, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
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
    if (flops) *flops = 3.0 * 2.0 * (double)n1 * (double)n2 * (double)w.dp;
    return launch_gram_tc(w.hi, w.lo, n1, n2, w.dp, w.kc, w.nchunk, w.Ppart,
                          reinterpret_cast<uint32_t *>(&w.scal[6]), (cudaStream_t)stream);
}

extern "C" rd_status cil_features(const float *d_X1, int64_t ld1, int64_t n1, const float *d_X2, int64_t ld2,
                                  int64_t n2, int64_t d, const double *d_radii_in, double b, int32_t M,
                                  double *d_radii_out, uint8_t *d_bins, int64_t *d_counts, double *d_C,
                                  int64_t *d_n_rechecked, void *d_work, size_t work_bytes, void *stream) {
    return cil_run(d_X1, ld1, n1, d_X2, ld2, n2, d, d_radii_in, b, M, d_radii_out, d_bins, d_counts, d_C,
                   d_n_rechecked, d_work, work_bytes, stream, false);
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
