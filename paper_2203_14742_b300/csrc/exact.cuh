// Exact squared distance of two FP32 vectors (Sec. 2.1, eq. eCDF).
//
// The paper defines the pattern distance on the reals.  The library's value
// of d2 is the real number S = sum_t (x_t - y_t)^2 of the FP32 inputs,
// rounded once to the nearest double (ties to even): it depends on no
// evaluation order, so any split of the work gives the same bits.
//
// It is formed in integer arithmetic.  A finite float is m 2^e with an
// integer 0 <= m < 2^24 and e = max(E, 1) - 150 >= -149 (E the biased
// exponent field), so each term x^2 + y^2 - 2xy is three integers below
// 2^48 placed at powers of two no smaller than 2^-298.  Every thread adds
// its terms into its own fixed-point accumulator N (unit 2^-298): XD digits
// of base 2^32, each held in a 64-bit signed integer in shared memory so
// that carries can wait.  A piece P 2^pos (P < 2^48) touches three digits,
// each receiving less than 2^32 in magnitude; the block then adds the
// threads' digits (integer sums: the order does not matter), and one
// thread propagates the carries and rounds N 2^-298 to 53 bits.
//
// Sizes: the largest piece is 2^48 at position 2 * 104 + 1 + 298 = 507, so
// N < 2^(555 + log2(3 d)); 19 digits (608 bits) hold it for d < 2^28, and a
// digit sum of the whole block stays below 3 d 2^32 < 2^63.
#pragma once
#include <cstdint>

namespace rdcil {

constexpr int XD = 19;                     // base-2^32 digits of the accumulator
constexpr int XD_BIAS = 298;               // the accumulator counts units of 2^-298
constexpr int64_t XD_MAX_D = 1ll << 28;    // longest vector the digit bounds allow

// a[k * stride] += (neg ? -1 : 1) * P 2^pos, pos >= 0, P < 2^48
__device__ __forceinline__ void xd_piece(long long *a, int stride, unsigned long long P, int pos, bool neg) {
    const int k = pos >> 5, r = pos & 31;
    const unsigned long long s = P << r;                        // low 64 bits of P 2^r
    long long v0 = (long long)(s & 0xffffffffull);
    long long v1 = (long long)(s >> 32);
    long long v2 = r ? (long long)(P >> (64 - r)) : 0ll;       // bits 64 and up
    if (neg) {
        v0 = -v0;
        v1 = -v1;
        v2 = -v2;
    }
    a[k * stride] += v0;
    a[(k + 1) * stride] += v1;
    a[(k + 2) * stride] += v2;
}

// a += x^2 + y^2 - 2 x y exactly; false when x or y is not finite
__device__ __forceinline__ bool xd_term(long long *a, int stride, float x, float y) {
    const unsigned ux = __float_as_uint(x), uy = __float_as_uint(y);
    const int Ex = (int)((ux >> 23) & 0xffu), Ey = (int)((uy >> 23) & 0xffu);
    const unsigned long long mx = (ux & 0x7fffffu) | (Ex ? 0x800000u : 0u);
    const unsigned long long my = (uy & 0x7fffffu) | (Ey ? 0x800000u : 0u);
    const int ex = max(Ex, 1) - 150, ey = max(Ey, 1) - 150;
    xd_piece(a, stride, mx * mx, 2 * ex + XD_BIAS, false);
    xd_piece(a, stride, my * my, 2 * ey + XD_BIAS, false);
    xd_piece(a, stride, mx * my, ex + ey + 1 + XD_BIAS, ((ux ^ uy) >> 31) == 0u);   // -2xy < 0 for equal signs
    return Ex != 0xff && Ey != 0xff;
}

// N 2^-298 rounded to the nearest double, ties to even, from the digit sums
// S[0..XD-1] (N = sum S[k] 2^(32 k) >= 0).
__device__ inline double xd_round(const long long *S) {
    unsigned dig[XD + 2];
    long long carry = 0;
#pragma unroll
    for (int k = 0; k < XD; ++k) {
        const long long t = S[k] + carry;
        dig[k] = (unsigned)(t & 0xffffffffll);
        carry = t >> 32;                       // arithmetic: floor division
    }
    dig[XD] = dig[XD + 1] = 0u;
    if (carry != 0) return __longlong_as_double(0x7ff8000000000000ll);   // not reached for S >= 0
    int top = XD - 1;
    while (top >= 0 && dig[top] == 0u) --top;
    if (top < 0) return 0.0;
    const int p = 32 * top + 31 - __clz(dig[top]);   // highest set bit
    if (p <= 52) {                                    // N < 2^53: exact
        const unsigned long long n = ((unsigned long long)dig[1] << 32) | dig[0];
        return __dmul_rn((double)n, 0x1p-298);
    }
    const int low = p - 52, k = low >> 5, r = low & 31;   // bits low .. p are kept
    const unsigned long long w0 = ((unsigned long long)dig[k + 1] << 32) | dig[k];
    const unsigned long long w1 = dig[k + 2];
    unsigned long long mant = ((w0 >> r) | (r ? (w1 << (64 - r)) : 0ull)) & ((1ull << 53) - 1ull);
    const int hb = low - 1;                               // the half-way bit
    const bool half = ((dig[hb >> 5] >> (hb & 31)) & 1u) != 0u;
    bool sticky = (dig[hb >> 5] & ((1u << (hb & 31)) - 1u)) != 0u;
    for (int i = 0; i < (hb >> 5); ++i) sticky |= dig[i] != 0u;
    int e = low - XD_BIAS;                                // value = mant 2^e
    if (half && (sticky || (mant & 1ull))) {
        ++mant;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            ++e;
        }
    }
    // always a normal double: 2^-298 <= value < 2^310
    const unsigned long long bits = ((unsigned long long)(e + 52 + 1023) << 52) | (mant - (1ull << 52));
    return __longlong_as_double((long long)bits);
}

// Shared memory of xd_block: XD digits per thread, XD per warp and the
// block's XD totals.
template <int NT>
struct XdShared {
    long long acc[XD * NT];
    long long wsum[XD * (NT / 32)];
    long long tot[XD];
    double wmax[NT / 32];
    int bad;
};

// The block's digit totals into sh.tot (every thread calls it after adding
// its terms into sh.acc; sh.tot valid in every thread on return).  The XD
// warp reductions are unrolled so their shuffle chains overlap, and thread
// k < XD adds digit k over the warps: integer sums, so no order matters.
template <int NT>
__device__ __forceinline__ void xd_reduce(XdShared<NT> &sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long v[XD];
#pragma unroll
    for (int k = 0; k < XD; ++k) v[k] = sh.acc[k * NT + tid];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < XD; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < XD; ++k) sh.wsum[k * (NT / 32) + warp] = v[k];
    __syncthreads();
    if (tid < XD) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += sh.wsum[tid * (NT / 32) + w];
        sh.tot[tid] = t;
    }
    __syncthreads();
}

// The digit sums of x[0..d) and y[0..d) (every thread of the block calls
// it): on return sh.tot[0..XD-1] holds the exact integer N of the
// segment's terms, sum tot[k] 2^(32 k), unnormalised, so the sums of
// several segments add digit by digit in any order (each stays below
// 3 d_total 2^32 < 2^63 for d_total < 2^28).  Returns false (in every
// thread) when an element is not finite.  The caller synchronises the
// block after reading sh.tot and before its next call.
template <int NT>
__device__ bool xd_block_digits(const float *__restrict__ x, const float *__restrict__ y, int64_t d,
                                XdShared<NT> &sh) {
    const int tid = threadIdx.x;
    long long *a = sh.acc + tid;
#pragma unroll
    for (int k = 0; k < XD; ++k) a[k * NT] = 0ll;
    if (tid == 0) sh.bad = 0;
    bool ok = true;
    for (int64_t t = tid; t < d; t += NT) ok &= xd_term(a, NT, __ldg(x + t), __ldg(y + t));
    __syncthreads();   // sh.bad cleared before any thread sets it
    if (!ok) sh.bad = 1;
    xd_reduce<NT>(sh);
    return sh.bad == 0;
}

// d2 of x[0..d) and y[0..d) by a whole block of NT threads (every thread
// calls it); with MAX also max_t |fl64(x_t - y_t)| (the FP64 difference
// rounded to nearest).  Results valid in thread 0; d2 is NaN when an
// element is not finite.
template <int NT, bool MAX>
__device__ double xd_block(const float *__restrict__ x, const float *__restrict__ y, int64_t d, XdShared<NT> &sh,
                           double *mx_out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long *a = sh.acc + tid;
#pragma unroll
    for (int k = 0; k < XD; ++k) a[k * NT] = 0ll;
    if (tid == 0) sh.bad = 0;
    bool ok = true;
    double mx = 0.0;
    for (int64_t t = tid; t < d; t += NT) {
        const float xv = __ldg(x + t), yv = __ldg(y + t);
        ok &= xd_term(a, NT, xv, yv);
        if (MAX) mx = fmax(mx, fabs(__dsub_rn((double)xv, (double)yv)));
    }
    __syncthreads();   // sh.bad cleared before any thread sets it
    if (!ok) sh.bad = 1;
    if (MAX) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) sh.wmax[warp] = mx;
    }
    xd_reduce<NT>(sh);
    double r = 0.0;
    if (tid == 0) {
        long long S[XD];
#pragma unroll
        for (int k = 0; k < XD; ++k) S[k] = sh.tot[k];
        r = sh.bad ? __longlong_as_double(0x7ff8000000000000ll) : xd_round(S);
        if (MAX) {
            double m = 0.0;
            for (int w = 0; w < NT / 32; ++w) m = fmax(m, sh.wmax[w]);
            *mx_out = m;
        }
    }
    __syncthreads();   // the shared arrays may be reused by the next call
    return r;
}

}  // namespace rdcil
