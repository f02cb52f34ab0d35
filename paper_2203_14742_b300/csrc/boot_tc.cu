// Bootstrap counts of the correlation integral on the tensor cores.
//
// Paper (arXiv 2203.14742): resampling with replacement of both pattern
// sets, Alg. 5 step 2.1 and Alg. 6 steps 2.1-2.2 (appendix A); the counts
// of eq. (CIL) of every resampled set pair.
//
// Resample t draws set-1 indices I_t(a) (a < n1) and set-2 indices J_t(b)
// (b < n2).  With the multiplicities c1[i][t] = #{a : I_t(a) = i} and
// c2[j][t] = #{b : J_t(b) = j} the count of radius k is the bilinear form
//   Y[t][k-1] = sum_a sum_b [K_{I(a) J(b)} >= k]
//             = sum_i c1[i][t] sum_j A_k[i][j] c2[j][t],   A_k = [K >= k],
// i.e. for every k the diagonal of C1^T A_k C2.  Z_k = A_k C2 is a dense
// product with 0/1 entries on one side and small integers on the other:
// bf16 holds both exactly (multiplicities up to 256), every product and
// every partial sum is an integer below 2^24 (a row of Z sums to at most
// sum_j c2[j][t] = n2), so FP32 accumulation in tensor memory is exact in
// any order.  The contraction with c1 and the sum over i are integer.
//
//   boot_count_kernel   multiplicities by integer atomics (one CTA per
//                       (resample, problem))
//   boot_prep_kernel    bins clamped to M and padded to [n1p][n2p], C2 as
//                       bf16 rows [t][j]
//                       (flags a multiplicity above 256), C1 transposed to
//                       [i][t]
//   bootstrap_tc_kernel one CTA per (problem, feature, 128-row tile,
//                       N tile of resamples, group of radii, K segment):
//                       per 64-column chunk TMA brings the C2 tile (issued
//                       one chunk ahead) and the threads build the 0/1
//                       tiles of the CTA's radii, both in 128-byte swizzled
//                       shared memory (two stages), one thread
//                       issues tcgen05.mma (M = 128, N = resamples of the
//                       tile, K = 16) into one TMEM accumulator per radius;
//                       the epilogue reads Z back with tcgen05.ld,
//                       multiplies by c1 (int32), sums over the 128 rows
//                       with a warp transpose-reduce and shared atomics,
//                       and adds into Y with 64-bit atomics.
// If a multiplicity exceeds 256 (probability below 1e-500 per resample, but
// possible) the tensor-core kernel does nothing and the SIMT bootstrap
// kernel, launched after it, counts instead.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <mutex>
#include "common.cuh"
#include "tc.cuh"

namespace rdcil {

static constexpr int BT_ROWS = 128, BT_K = 64, BT_KG_MAX = 4, BT_THREADS = 128;
static constexpr int BT_A_BYTES = BT_ROWS * BT_K * 2;   // one 0/1 tile, bf16, 16 KiB

struct BootDims {
    int64_t n1, n2, n1p, n2p;
    int T, Tn, TnA, NT, Tp, M, KG, G, nf, P, MT;
};

static inline int64_t rup64(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

static BootDims boot_dims(int64_t n1, int64_t n2, int M, int T, int nf, int P) {
    BootDims d{};
    d.n1 = n1;
    d.n2 = n2;
    d.n1p = rup64(n1, BT_ROWS);
    d.n2p = rup64(n2, BT_K);
    d.T = T;
    d.NT = (T + 255) / 256;
    const int per = (T + d.NT - 1) / d.NT;
    d.Tn = (int)rup64(per, 16);
    d.Tp = d.NT * d.Tn;
    d.TnA = (int)rup64(d.Tn, 32);
    d.M = M;
    d.KG = 512 / d.TnA;
    if (d.KG > BT_KG_MAX) d.KG = BT_KG_MAX;
    if (d.KG > M) d.KG = M;
    d.G = (M + d.KG - 1) / d.KG;
    d.nf = nf;
    d.P = P;
    d.MT = (int)(d.n1p / BT_ROWS);
    return d;
}

struct BootWork {
    BootDims d;
    uint8_t *BP;        // [P][nf][n1p][n2p] bins, zero padded
    uint16_t *C2;       // [P][Tp][n2p] bf16 multiplicities of set 2
    uint16_t *C1T;      // [P][n1p][Tp] multiplicities of set 1
    uint32_t *C1cnt;    // [P][Tp][n1p]
    uint32_t *C2cnt;    // [P][Tp][n2p]
    uint32_t *flag;     // [0] a multiplicity above 256, [1] tensor-core wait timed out
    size_t cnt_bytes;   // C1cnt .. flag, cleared per call
    size_t bytes;
};

static BootWork boot_layout(const BootDims &d, void *base) {
    BootWork w{};
    w.d = d;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)rup64((int64_t)(off + bytes), 256);
        return (char *)base + o;
    };
    const int64_t P = d.P;
    w.BP = (uint8_t *)take((size_t)(P * d.nf * d.n1p * d.n2p));
    w.C2 = (uint16_t *)take(sizeof(uint16_t) * (size_t)(P * d.Tp * d.n2p));
    w.C1T = (uint16_t *)take(sizeof(uint16_t) * (size_t)(P * d.n1p * d.Tp) + 64);   // + the 32-value read past a row
    const size_t c0 = off;
    w.C1cnt = (uint32_t *)take(sizeof(uint32_t) * (size_t)(P * d.Tp * d.n1p));
    w.C2cnt = (uint32_t *)take(sizeof(uint32_t) * (size_t)(P * d.Tp * d.n2p));
    w.flag = (uint32_t *)take(sizeof(uint32_t) * 2);
    w.cnt_bytes = off - c0;
    w.bytes = off;
    return w;
}

__device__ __forceinline__ uint32_t boot_index(uint64_t seed, uint64_t ctr, uint32_t n) {
    return (uint32_t)__umul64hi(splitmix64_at(seed, ctr), (uint64_t)n);
}

__global__ void boot_count_kernel(BootWork w, uint64_t seed) {
    const BootDims &d = w.d;
    const int t = blockIdx.x, p = blockIdx.y;
    const uint64_t sp = seed + (uint64_t)p;
    uint32_t *c1 = w.C1cnt + ((int64_t)p * d.Tp + t) * d.n1p;
    uint32_t *c2 = w.C2cnt + ((int64_t)p * d.Tp + t) * d.n2p;
    for (int a = threadIdx.x; a < (int)d.n1; a += blockDim.x)
        atomicAdd(&c1[boot_index(sp, (((uint64_t)t * 2u + 0u) << 32) | (uint64_t)a, (uint32_t)d.n1)], 1u);
    for (int b = threadIdx.x; b < (int)d.n2; b += blockDim.x)
        atomicAdd(&c2[boot_index(sp, (((uint64_t)t * 2u + 1u) << 32) | (uint64_t)b, (uint32_t)d.n2)], 1u);
}

__global__ void boot_prep_kernel(BootWork w, const uint8_t *__restrict__ bins, uint32_t mult_limit) {
    const BootDims &d = w.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // bins clamped to M (which leaves every [K >= k], k <= M, unchanged and
    // keeps the byte-wise compare below carry-free), zero padded (K = 0
    // counts under no radius)
    const int64_t nb = (int64_t)d.P * d.nf * d.n1p * d.n2p;
    for (int64_t e = e0; e < nb; e += stride) {
        const int64_t j = e % d.n2p, r = e / d.n2p;
        const int64_t i = r % d.n1p, pf = r / d.n1p;
        const int K = (i < d.n1 && j < d.n2) ? (int)bins[(pf * d.n1 + i) * d.n2 + j] : 0;
        w.BP[e] = (uint8_t)min(K, d.M);
    }
    // C2 rows as bf16 (exact up to 256)
    const int64_t nc2 = (int64_t)d.P * d.Tp * d.n2p;
    for (int64_t e = e0; e < nc2; e += stride) {
        const uint32_t v = w.C2cnt[e];
        if (v > mult_limit) atomicOr(&w.flag[0], 1u);
        // an integer up to 256 has at most 8 significant bits: the upper half
        // of its FP32 pattern is its bf16 pattern exactly
        w.C2[e] = (uint16_t)(__float_as_uint((float)v) >> 16);
    }
    // C1 transposed to [i][t]
    const int64_t nc1 = (int64_t)d.P * d.n1p * d.Tp;
    for (int64_t e = e0; e < nc1; e += stride) {
        const int64_t t = e % d.Tp, r = e / d.Tp;
        const int64_t i = r % d.n1p, p = r / d.n1p;
        w.C1T[e] = (uint16_t)w.C1cnt[(p * d.Tp + t) * d.n1p + i];
    }
}

// byte offset of 16-byte chunk ch (0..7) of row r in a K-major tile with
// the 128-byte swizzle (8-row groups of 1024 bytes)
__device__ __forceinline__ uint32_t sw128_off(int r, int ch) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4));
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 0/1 bf16 flags (K >= k) of 8 bins bytes (two words) as one 16-byte chunk
__device__ __forceinline__ uint4 ge_flags(uint32_t w0, uint32_t w1, uint32_t add) {
    // byte-wise K + 0x80 - k: bit 7 set iff K >= k (K <= 32, 1 <= k <= 32:
    // no carry leaves a byte)
    const uint32_t m0 = ((w0 + add) >> 7) & 0x01010101u, m1 = ((w1 + add) >> 7) & 0x01010101u;
    uint4 o;
    o.x = __byte_perm(m0, 0u, 0x4140) * 0x3F80u;   // bf16 1.0 = 0x3F80
    o.y = __byte_perm(m0, 0u, 0x4342) * 0x3F80u;
    o.z = __byte_perm(m1, 0u, 0x4140) * 0x3F80u;
    o.w = __byte_perm(m1, 0u, 0x4342) * 0x3F80u;
    return o;
}

__global__ void __launch_bounds__(BT_THREADS, 1)
bootstrap_tc_kernel(const __grid_constant__ CUtensorMap tm_c2, BootWork w, int S, unsigned long long *__restrict__ Y,
                    uint32_t spin) {
    const BootDims &d = w.d;
    if (*(volatile uint32_t *)w.flag) return;   // the SIMT kernel counts instead
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = d.KG * BT_A_BYTES + d.Tn * 128;
    // [0, 1] stage consumed (MMA commit), [2] all MMAs done, [3, 4] the stage's
    // C2 tile landed (TMA)
    uint64_t *bar = (uint64_t *)(smem + 2 * stage_bytes);
    uint32_t *tslot = (uint32_t *)(bar + 5);
    __shared__ int sY[BT_KG_MAX * 256];
    __shared__ int s_fail;

    int idx = blockIdx.x;
    const int seg = idx % S; idx /= S;
    const int g = idx % d.G; idx /= d.G;
    const int ni = idx % d.NT; idx /= d.NT;
    const int mi = idx % d.MT; idx /= d.MT;
    const int f = idx % d.nf;
    const int p = idx / d.nf;
    const int k0 = g * d.KG + 1;
    const int kn = min(d.KG, d.M - g * d.KG);
    const int nch = (int)(d.n2p / BT_K);
    const int c_lo = (int)((int64_t)seg * nch / S), c_hi = (int)((int64_t)(seg + 1) * nch / S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tensor-memory columns: the accumulators of the CTA's radii, rounded up
    // to a power of two (at least 32)
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(d.KG * d.TnA)) ncols <<= 1;

    for (int e = tid; e < BT_KG_MAX * 256; e += BT_THREADS) sY[e] = 0;
    if (tid == 0) {
        for (int q = 0; q < 5; ++q) mbar_init(&bar[q], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    const int64_t i = (int64_t)mi * BT_ROWS + tid;   // this thread's row of the tile
    const uint8_t *brow = w.BP + (((int64_t)p * d.nf + f) * d.n1p + i) * d.n2p;
    const int trow = p * d.Tp + ni * d.Tn;           // first C2 row of the resample tile (TMA y)
    const uint32_t idesc = idesc_bf16_f32(BT_ROWS, d.Tn);
    const uint32_t c2_bytes = (uint32_t)d.Tn * 128u;
    const int nloc = c_hi - c_lo;
    int issued = 0, landed = 0;   // TMA copies issued / seen complete (thread 0)
    if (tid == 0 && nloc > 0) {
        mbar_expect_tx(&bar[3], c2_bytes);
        tma_load_2d(smem + d.KG * BT_A_BYTES, &tm_c2, c_lo * BT_K, trow, &bar[3]);
        issued = 1;
    }
    uint4 bw[4];
    if (nloc > 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) bw[q] = *reinterpret_cast<const uint4 *>(brow + (int64_t)c_lo * BT_K + q * 16);
    }
    bool failed = false;
    for (int lc = 0; lc < nloc; ++lc) {
        const int c = c_lo + lc, st = lc & 1;
        bool ok = s_fail == 0;
        if (ok && lc >= 2) ok = mbar_wait(&bar[st], (uint32_t)((lc - 2) >> 1) & 1u, spin);
        if (__syncthreads_or(ok ? 0 : 1)) { failed = true; break; }
        uint8_t *sb = smem + st * stage_bytes;
        // next chunk's bins, then this chunk's 0/1 tiles, one per radius
        uint4 bn[4];
        if (lc + 1 < nloc) {
#pragma unroll
            for (int q = 0; q < 4; ++q) bn[q] = *reinterpret_cast<const uint4 *>(brow + (int64_t)(c + 1) * BT_K + q * 16);
        }
        for (int kk = 0; kk < kn; ++kk) {
            const uint32_t add = (uint32_t)(0x80 - (k0 + kk)) * 0x01010101u;
            uint8_t *at = sb + kk * BT_A_BYTES;
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
                const uint4 q = bw[ch >> 1];
                const uint4 o = (ch & 1) ? ge_flags(q.z, q.w, add) : ge_flags(q.x, q.y, add);
                *reinterpret_cast<uint4 *>(at + sw128_off(tid, ch)) = o;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(&bar[3 + st], (uint32_t)(lc >> 1) & 1u, spin)) {
                s_fail = 1;
            } else {
                landed = lc + 1;
                fence_after();
                const uint32_t bB = smem_u32(sb + d.KG * BT_A_BYTES);
                for (int kk = 0; kk < kn; ++kk) {
                    const uint32_t bA = smem_u32(sb + kk * BT_A_BYTES);
#pragma unroll
                    for (int ks = 0; ks < BT_K / 16; ++ks)
                        mma_bf16(tmem + (uint32_t)(kk * d.TnA), smem_desc_sw128(bA + ks * 32),
                                 smem_desc_sw128(bB + ks * 32), idesc, (lc == 0 && ks == 0) ? 0u : 1u);
                }
                mma_commit(&bar[st]);
                // the next chunk's C2 tile into the other stage, once the MMAs
                // of the chunk before this one have read it
                if (lc + 1 < nloc) {
                    const int sn = (lc + 1) & 1;
                    if (lc >= 1 && !mbar_wait(&bar[sn], (uint32_t)((lc - 1) >> 1) & 1u, spin)) {
                        s_fail = 1;
                    } else {
                        mbar_expect_tx(&bar[3 + sn], c2_bytes);
                        tma_load_2d(smem + sn * stage_bytes + d.KG * BT_A_BYTES, &tm_c2, (c + 1) * BT_K, trow,
                                    &bar[3 + sn]);
                        issued = lc + 2;
                    }
                }
            }
        }
        if (lc + 1 < nloc) {
#pragma unroll
            for (int q = 0; q < 4; ++q) bw[q] = bn[q];
        }
    }
    if (tid == 0) {
        // copies still in flight land before the shared memory is released
        for (int it = landed; it < issued; ++it) mbar_wait(&bar[3 + (it & 1)], (uint32_t)(it >> 1) & 1u, spin);
    }
    // every MMA issued by this CTA completes before its tensor memory is
    // read or released
    if (tid == 0) {
        mma_commit(&bar[2]);
        if (!mbar_wait(&bar[2], 0, spin)) s_fail = 1;
    }
    __syncthreads();
    const bool bad = failed || s_fail;
    fence_after();
    if (!bad && c_hi > c_lo) {
        const uint32_t lrow = (uint32_t)(warp * 32) << 16;
        const uint16_t *c1row = w.C1T + ((int64_t)p * d.n1p + (int64_t)mi * BT_ROWS + warp * 32 + lane) * d.Tp +
                                (int64_t)ni * d.Tn;
        for (int kk = 0; kk < kn; ++kk) {
            for (int tb = 0; tb < d.Tn; tb += 32) {
                // this row's 32 multiplicities (64 bytes, 16-byte aligned)
                uint32_t cw[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(c1row + tb + 8 * q);
                    cw[4 * q] = u.x; cw[4 * q + 1] = u.y; cw[4 * q + 2] = u.z; cw[4 * q + 3] = u.w;
                }
                float z[32];
                tmem_ld32(tmem + lrow + (uint32_t)(kk * d.TnA + tb), z);
                int v[32];
#pragma unroll
                for (int l = 0; l < 32; ++l) {
                    const int c1 = (tb + l < d.Tn) ? (int)((cw[l >> 1] >> (16 * (l & 1))) & 0xFFFFu) : 0;
                    v[l] = c1 ? __float2int_rn(z[l]) * c1 : 0;
                }
                // transpose-reduce: afterwards lane l holds column tb + l summed
                // over the warp's 32 rows
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const bool upper = (lane & s) != 0;
#pragma unroll
                    for (int q = 0; q < s; ++q) {
                        const int send = upper ? v[q] : v[q + s];
                        const int keep = upper ? v[q + s] : v[q];
                        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
                    }
                }
                if (tb + lane < d.Tn && v[0]) atomicAdd(&sY[kk * d.Tn + tb + lane], v[0]);
            }
        }
    }
    __syncthreads();
    if (!bad) {
        const int Mt = d.nf * d.M;
        for (int e = tid; e < kn * d.Tn; e += BT_THREADS) {
            const int kk = e / d.Tn, tl = e - kk * d.Tn;
            const int t = ni * d.Tn + tl;
            if (t < d.T && sY[e])
                atomicAdd(&Y[((int64_t)p * d.T + t) * Mt + f * d.M + (k0 - 1 + kk)], (unsigned long long)sY[e]);
        }
    } else if (tid == 0) {
        atomicOr(&w.flag[1], 1u);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

static PFN_cuTensorMapEncodeTiled_v12000 boot_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) ==
                cudaSuccess &&
            r == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)q;
    });
    return fn;
}

// multiplicities above this send the counting to the SIMT kernel (256: the
// largest bf16 holds every integer up to it; lower only to test that path)
static uint32_t g_mult_limit = 256;
void boot_set_mult_limit(int n) { g_mult_limit = (n < 1 || n > 256) ? 256u : (uint32_t)n; }

size_t boot_workspace_bytes(int64_t n1, int64_t n2, int M, int T, int nf, int P) {
    return boot_layout(boot_dims(n1, n2, M, T, nf, P), nullptr).bytes;
}

// Counts Y (cleared by the caller) on the tensor cores; *flag_out = the
// workspace's flag words ([0] multiplicity above 256: the caller's SIMT
// kernel must count; [1] a bounded wait gave up).
rd_status launch_bootstrap_tc(const uint8_t *bins, int nf, int64_t n1, int64_t n2, int M, int T, uint64_t seed,
                              int P, int64_t *Y, void *work, size_t work_bytes, const uint32_t **flag_out,
                              cudaStream_t s) {
    const BootDims d = boot_dims(n1, n2, M, T, nf, P);
    BootWork w = boot_layout(d, work);
    if (w.bytes > work_bytes || (((uintptr_t)work) & 255)) return RD_ERR_INVALID_ARG;
    RD_CUDA_TRY(cudaMemsetAsync(w.C1cnt, 0, w.cnt_bytes, s));
    boot_count_kernel<<<dim3((unsigned)T, (unsigned)P), 256, 0, s>>>(w, seed);
    note_launch();
    boot_prep_kernel<<<4 * 148, 256, 0, s>>>(w, bins, g_mult_limit);
    note_launch();
    // units of work; K segments to give every SM about one CTA
    const int64_t units = (int64_t)P * nf * d.MT * d.NT * d.G;
    const int nch = (int)(d.n2p / BT_K);
    int S = units >= 148 ? 1 : (int)(148 / units);
    if (S > nch) S = nch;
    if (S < 1) S = 1;
    if (units * S > 0x7FFFFFFF) return RD_ERR_UNSUPPORTED;
    const size_t smem = 1024 + 2 * (size_t)(d.KG * BT_A_BYTES + d.Tn * 128) + 64;
    // C2 as a 2-D tensor: n2p bf16 columns (inner) x P Tp rows; boxes of 64
    // columns (128 bytes, the swizzle span) x Tn resamples
    auto enc = boot_encode_fn();
    if (!enc) return RD_ERR_CUDA;
    CUtensorMap tm;
    cuuint64_t dims[2] = {(cuuint64_t)d.n2p, (cuuint64_t)((int64_t)P * d.Tp)};
    cuuint64_t strides[1] = {(cuuint64_t)d.n2p * 2};
    cuuint32_t box[2] = {(cuuint32_t)BT_K, (cuuint32_t)d.Tn};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, w.C2, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return RD_ERR_CUDA;
    // the size varies with the problem and the attribute is per device: set it per call
    RD_CUDA_TRY(cudaFuncSetAttribute(bootstrap_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    bootstrap_tc_kernel<<<(unsigned)(units * S), BT_THREADS, smem, s>>>(
        tm, w, S, reinterpret_cast<unsigned long long *>(Y), MBAR_WAIT_LIMIT);
    note_launch();
    *flag_out = w.flag;
    return cuda_status(cudaGetLastError());
}

}  // namespace rdcil
